// zq_node.cuh -- one node's transform applied to vectors, shared by the
// sweeps (zq_apply.cu) and the explicit generation of Q~ (zq_qgen.cu).
//
// Upward (Algorithm 2, Eqs. 4.2-4.3): with the children's Info-sets
// [t_x; r_x], [t_y; r_y],
//   t_p = alpha t_x + beta t_y,   s = beta t_x - alpha t_y,
//   [r_p; eps_p] = G [r_x?; r_y?; s]   (r_c only for internal children).
// Downward (Algorithm 3, Theorem 4.3, Eqs. 4.6-4.7): with p's Velocity-set
// [T; l] and residue coefficients w_p,
//   [a_x?; a_y?; sigma] = G^T [l; w_p],
//   L_x = [alpha T + beta sigma; a_x],  L_y = [beta T - alpha sigma; a_y].
// G is applied as its three Householder reflectors with the diagonal sign
// normalisation D (G u = D H3 H2 H1 u, G^T z = H1 H2 H3 D z) restricted to
// their possibly nonzero rows, or as the explicit 3 x 3 matrix for Case I
// (record layouts in zq_internal.cuh).
#pragma once

#include "zq_internal.cuh"

namespace zq {

namespace {

// How a record is read: through the read-only path (records no thread of
// the running kernel writes), or with coherent L2 loads (records written in
// the same launch).
constexpr int kLdNC = 0, kLdCG = 1;

// Load W words of a record (16-byte vector loads).
template <typename T, int W, int LD = kLdNC>
__device__ __forceinline__ void load_rec(const T* g, T (&r)[W]) {
  if constexpr (sizeof(T) == 4) {
    const float4* p = reinterpret_cast<const float4*>(g);
#pragma unroll
    for (int i = 0; i < W / 4; ++i) {
      const float4 q = LD == kLdNC ? __ldg(p + i) : __ldcg(p + i);
      r[4 * i] = q.x; r[4 * i + 1] = q.y; r[4 * i + 2] = q.z; r[4 * i + 3] = q.w;
    }
  } else {
    const double2* p = reinterpret_cast<const double2*>(g);
#pragma unroll
    for (int i = 0; i < W / 2; ++i) {
      const double2 q = LD == kLdNC ? __ldg(p + i) : __ldcg(p + i);
      r[2 * i] = q.x; r[2 * i + 1] = q.y;
    }
  }
}

template <typename T>
__device__ __forceinline__ void load6(const T* __restrict__ p, T* v) {
#pragma unroll
  for (int i = 0; i < 6; ++i) v[i] = p[i];
}

template <typename T>
__device__ __forceinline__ void store6(T* __restrict__ p, const T* v) {
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = v[i];
}

__device__ __forceinline__ bool sign_set(float x) { return __float_as_int(x) < 0; }
__device__ __forceinline__ bool sign_set(double x) { return __double2hiint(x) < 0; }

// One factor D_j H_j of G = (D_3 H_3)(D_2 H_2)(D_1 H_1): H_j = I - |tau| v v^T
// with v(j) = 1 and the other nonzeros of v at rows R[0..n-1] with values
// vv[0..n-1]; D_j negates entry j when tau's sign bit is set (the diagonal
// sign normalisation of T22).  TR = false: u <- D_j H_j u (forward);
// TR = true: u <- H_j D_j u (the transpose, G^T = H_1 D_1 H_2 D_2 H_3 D_3).
template <typename T, int NV, bool TR>
__device__ __forceinline__ void reflect(T* u, int j, const int (&R)[NV], const T* vv, T tau_s) {
  const bool neg = sign_set(tau_s);
  const T tau = neg ? -tau_s : tau_s;
  if (TR && neg) u[j] = -u[j];
  T w = u[j];
#pragma unroll
  for (int i = 0; i < NV; ++i) w += vv[i] * u[R[i]];
  w *= tau;
  u[j] -= w;
#pragma unroll
  for (int i = 0; i < NV; ++i) u[R[i]] -= w * vv[i];
  if (!TR && neg) u[j] = -u[j];
}

// G u and G^T u for the two Householder record types (layout in zq_internal.cuh).
template <typename T>
__device__ __forceinline__ void g6(const T* r, T* u, bool transpose) {
  constexpr int R0[2] = {4, 5}, R1[3] = {3, 4, 5}, R2[3] = {3, 4, 5};
  if (!transpose) {
    reflect<T, 2, false>(u, 0, R0, r + 5, r[2]);
    reflect<T, 3, false>(u, 1, R1, r + 7, r[3]);
    reflect<T, 3, false>(u, 2, R2, r + 10, r[4]);
  } else {
    reflect<T, 3, true>(u, 2, R2, r + 10, r[4]);
    reflect<T, 3, true>(u, 1, R1, r + 7, r[3]);
    reflect<T, 2, true>(u, 0, R0, r + 5, r[2]);
  }
}

template <typename T>
__device__ __forceinline__ void g9(const T* r, T* u, bool transpose) {
  constexpr int R0[3] = {3, 7, 8}, R1[5] = {3, 4, 6, 7, 8}, R2[6] = {3, 4, 5, 6, 7, 8};
  if (!transpose) {
    reflect<T, 3, false>(u, 0, R0, r + 5, r[2]);
    reflect<T, 5, false>(u, 1, R1, r + 8, r[3]);
    reflect<T, 6, false>(u, 2, R2, r + 13, r[4]);
  } else {
    reflect<T, 6, true>(u, 2, R2, r + 13, r[4]);
    reflect<T, 5, true>(u, 1, R1, r + 8, r[3]);
    reflect<T, 3, true>(u, 0, R0, r + 5, r[2]);
  }
}

// --------------------------------------------------------- node: upward
// X, Y: the children's Info-sets [t; r] (r unused for leaves).  Writes the
// node's Info-set to P and its residues to res.
template <typename T, int TYPE, int LD = kLdNC>
__device__ __forceinline__ void up_node(const T* recp, const T* X, const T* Y, bool xi,
                                        T* P, T* __restrict__ res) {
  T r[rec_words(TYPE)];
  load_rec<T, rec_words(TYPE), LD>(recp, r);
  const T al = r[0], be = r[1];
  T u[9];
  int k = 0;
  if (TYPE == 2) {
    u[0] = X[3]; u[1] = X[4]; u[2] = X[5];
    u[3] = Y[3]; u[4] = Y[4]; u[5] = Y[5];
    k = 6;
  } else if (TYPE == 1) {
    const T* C = xi ? X : Y;
    u[0] = C[3]; u[1] = C[4]; u[2] = C[5];
    k = 3;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    P[a] = al * X[a] + be * Y[a];
    u[k + a] = be * X[a] - al * Y[a];
  }
  if (TYPE == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) P[3 + i] = r[2 + 3 * i] * u[0] + r[3 + 3 * i] * u[1] + r[4 + 3 * i] * u[2];
    return;
  }
  if (TYPE == 1) {
    g6(r, u, false);
#pragma unroll
    for (int i = 0; i < 3; ++i) res[i] = u[3 + i];
  } else {
    g9(r, u, false);
#pragma unroll
    for (int i = 0; i < 6; ++i) res[i] = u[3 + i];
  }
  P[3] = u[0]; P[4] = u[1]; P[5] = u[2];
}

// ------------------------------------------------------- node: downward
template <typename T, int TYPE, int LD = kLdNC>
__device__ __forceinline__ void down_node(const T* recp, const T* Lp, const T* __restrict__ w,
                                          bool xi, T* Lx, T* Ly) {
  T r[rec_words(TYPE)];
  load_rec<T, rec_words(TYPE), LD>(recp, r);
  const T al = r[0], be = r[1];
  T z[9];
  z[0] = Lp[3]; z[1] = Lp[4]; z[2] = Lp[5];
  T sg[3];
  if (TYPE == 0) {
#pragma unroll
    for (int j = 0; j < 3; ++j) sg[j] = r[2 + j] * z[0] + r[5 + j] * z[1] + r[8 + j] * z[2];
  } else if (TYPE == 1) {
#pragma unroll
    for (int i = 0; i < 3; ++i) z[3 + i] = w[i];
    g6(r, z, true);
    T* c = xi ? Lx : Ly;
    c[3] = z[0]; c[4] = z[1]; c[5] = z[2];
    sg[0] = z[3]; sg[1] = z[4]; sg[2] = z[5];
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) z[3 + i] = w[i];
    g9(r, z, true);
    Lx[3] = z[0]; Lx[4] = z[1]; Lx[5] = z[2];
    Ly[3] = z[3]; Ly[4] = z[4]; Ly[5] = z[5];
    sg[0] = z[6]; sg[1] = z[7]; sg[2] = z[8];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Lx[i] = al * Lp[i] + be * sg[i];
    Ly[i] = be * Lp[i] - al * sg[i];
  }
}

}  // namespace

}  // namespace zq
