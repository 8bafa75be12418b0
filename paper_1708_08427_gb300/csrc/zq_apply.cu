// zq_apply.cu -- the two sweeps.
//
// Upward (Q~ v, Algorithm 2, Eqs. 4.2-4.3): a leaf's Info-set is its bead
// vector f_i (Definition 4.1); for node p with children x, y
//   t_p = alpha t_x + beta t_y,   s = beta t_x - alpha t_y,
//   [r_p; eps_p] = G [r_x?; r_y?; s]   (r_c only for internal children),
// eps_p (k - 3 numbers) is p's Residue, written at its residue offset.
// Downward (Q~^T w, Algorithm 3, Theorem 4.3, Eqs. 4.6-4.7): the root
// Velocity-set is 0; for node p with Velocity-set [T; l] and residue
// coefficients w_p
//   [a_x?; a_y?; sigma] = G^T [l; w_p],
//   L_x = [alpha T + beta sigma; a_x],  L_y = [beta T - alpha sigma; a_y],
// and a leaf's velocity is the first three entries of its Velocity-set.
//
// G is applied as its three Householder reflectors with the diagonal sign
// normalisation D = diag(+-1, +-1, +-1, 1, ...) (G u = D H3 H2 H1 u,
// G^T z = H1 H2 H3 D z) restricted to their possibly nonzero rows, or as the
// explicit 3 x 3 matrix for Case I.
//
// Schedule: heights 1..cut level by level over all bodies (records and
// Info-/Velocity-sets of a height are contiguous; one launch per height),
// the nodes above the cut one thread block per body.  Upward: levels then
// tails; downward: tails then levels.
#include "zq_internal.cuh"

namespace zq {

namespace {

constexpr int kThreads = 256;

template <typename T>
struct ApplyArgs {
  int64_t N;
  const int64_t* off;
  const int32_t* perm;
  const int2* sc;
  const int32_t* sroff;
  const uint8_t* sheight;
  const int32_t* sid;
  const int32_t* bstart;
  const int32_t* brec;
  const int32_t* root_slot;
  int cut;
  const T* rec;
  T* xs;        // Info-/Velocity-sets by slot [nodes * 6]
  const T* in;  // up: bead planes; down: residues
  T* out;       // up: residues; down: bead planes
};

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double2; };

// Load W words of a record (16-byte vector loads, read-only path).
template <typename T, int W>
__device__ __forceinline__ void load_rec(const T* __restrict__ g, T (&r)[W]) {
  if constexpr (sizeof(T) == 4) {
    const float4* p = reinterpret_cast<const float4*>(g);
#pragma unroll
    for (int i = 0; i < W / 4; ++i) {
      const float4 q = __ldg(p + i);
      r[4 * i] = q.x; r[4 * i + 1] = q.y; r[4 * i + 2] = q.z; r[4 * i + 3] = q.w;
    }
  } else {
    const double2* p = reinterpret_cast<const double2*>(g);
#pragma unroll
    for (int i = 0; i < W / 2; ++i) {
      const double2 q = __ldg(p + i);
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

template <typename T>
__device__ __forceinline__ void load_bead(const ApplyArgs<T>& a, int32_t code, T* t) {
  const int32_t i = a.perm[leaf_pos(code)];
  t[0] = a.in[i];
  t[1] = a.in[a.N + i];
  t[2] = a.in[2 * a.N + i];
}

template <typename T>
__device__ __forceinline__ void store_bead(const ApplyArgs<T>& a, int32_t code, const T* L) {
  const int32_t i = a.perm[leaf_pos(code)];
  a.out[i] = L[0];
  a.out[a.N + i] = L[1];
  a.out[2 * a.N + i] = L[2];
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
template <typename T, int TYPE>
__device__ __forceinline__ void up_node(const T* __restrict__ recp, const T* X, const T* Y, bool xi,
                                        T* P, T* __restrict__ res) {
  T r[rec_words(TYPE)];
  load_rec<T, rec_words(TYPE)>(recp, r);
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
template <typename T, int TYPE>
__device__ __forceinline__ void down_node(const T* __restrict__ recp, const T* Lp, const T* __restrict__ w,
                                          bool xi, T* Lx, T* Ly) {
  T r[rec_words(TYPE)];
  load_rec<T, rec_words(TYPE)>(recp, r);
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

template <typename T, int TYPE>
__device__ __forceinline__ void up_slot(const ApplyArgs<T>& a, int64_t s, int64_t rw) {
  const int2 cc = a.sc[s];
  T X[6], Y[6], P[6];
  if (is_leaf(cc.x)) load_bead(a, cc.x, X); else load6(a.xs + (int64_t)cc.x * 6, X);
  if (is_leaf(cc.y)) load_bead(a, cc.y, Y); else load6(a.xs + (int64_t)cc.y * 6, Y);
  up_node<T, TYPE>(a.rec + rw, X, Y, cc.x >= 0, P, a.out + a.sroff[s]);
  store6(a.xs + s * 6, P);
}

template <typename T, int TYPE>
__device__ __forceinline__ void down_slot(const ApplyArgs<T>& a, int64_t s, int64_t rw, const T* Lp) {
  const int2 cc = a.sc[s];
  T Lx[6], Ly[6];
  down_node<T, TYPE>(a.rec + rw, Lp, a.in + a.sroff[s], cc.x >= 0, Lx, Ly);
  if (is_leaf(cc.x)) store_bead(a, cc.x, Lx); else store6(a.xs + (int64_t)cc.x * 6, Lx);
  if (is_leaf(cc.y)) store_bead(a, cc.y, Ly); else store6(a.xs + (int64_t)cc.y * 6, Ly);
}

// ------------------------------------------------------------- kernels
template <typename T>
__global__ void __launch_bounds__(kThreads) k_up_level(ApplyArgs<T> a, int h) {
  const int b0 = 3 * (h - 1);
  const int32_t s0 = a.bstart[b0], s1 = a.bstart[b0 + 1], s2 = a.bstart[b0 + 2], s3 = a.bstart[b0 + 3];
  const int32_t r0 = a.brec[b0], r1 = a.brec[b0 + 1], r2 = a.brec[b0 + 2];
  for (int64_t s = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < s3;
       s += (int64_t)gridDim.x * blockDim.x) {
    if (s < s1) up_slot<T, 0>(a, s, r0 + (s - s0) * rec_words(0));
    else if (s < s2) up_slot<T, 1>(a, s, r1 + (s - s1) * rec_words(1));
    else up_slot<T, 2>(a, s, r2 + (s - s2) * rec_words(2));
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_down_level(ApplyArgs<T> a, int h) {
  const int b0 = 3 * (h - 1);
  const int32_t s0 = a.bstart[b0], s1 = a.bstart[b0 + 1], s2 = a.bstart[b0 + 2], s3 = a.bstart[b0 + 3];
  const int32_t r0 = a.brec[b0], r1 = a.brec[b0 + 1], r2 = a.brec[b0 + 2];
  for (int64_t s = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < s3;
       s += (int64_t)gridDim.x * blockDim.x) {
    T Lp[6];
    load6(a.xs + s * 6, Lp);
    if (s < s1) down_slot<T, 0>(a, s, r0 + (s - s0) * rec_words(0), Lp);
    else if (s < s2) down_slot<T, 1>(a, s, r1 + (s - s1) * rec_words(1), Lp);
    else down_slot<T, 2>(a, s, r2 + (s - s2) * rec_words(2), Lp);
  }
}

template <typename T>
__device__ __forceinline__ void tail_range(const ApplyArgs<T>& a, int32_t j, int32_t* lo, int32_t* hi) {
  const int bt = 3 * a.cut;
  id_range(a.sid, a.bstart[bt], a.bstart[bt + 1], a.off[j] - j, a.off[j + 1] - (j + 1), lo, hi);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_up_tail(ApplyArgs<T> a) {
  const int32_t j = blockIdx.x;
  int32_t lo, hi;
  tail_range(a, j, &lo, &hi);
  if (lo == hi) return;
  const int bt = 3 * a.cut;
  const int32_t t0 = a.bstart[bt], rt = a.brec[bt];
  const int H = a.sheight[a.root_slot[j]];
  for (int h = a.cut + 1; h <= H; ++h) {
    for (int32_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
      if (a.sheight[s] != h) continue;
      const int2 cc = a.sc[s];
      const int64_t rw = rt + (int64_t)(s - t0) * kRecMax;
      const int type = (cc.x >= 0) + (cc.y >= 0);
      if (type == 0) up_slot<T, 0>(a, s, rw);
      else if (type == 1) up_slot<T, 1>(a, s, rw);
      else up_slot<T, 2>(a, s, rw);
    }
    __syncthreads();
  }
}

// Runs before the levels: zero root Velocity-set for every body (Q~^T
// only), then the nodes above the cut from the root down.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_down_tail(ApplyArgs<T> a) {
  const int32_t j = blockIdx.x;
  const int32_t rs = a.root_slot[j];
  if (threadIdx.x < 6) a.xs[(int64_t)rs * 6 + threadIdx.x] = T(0);
  __syncthreads();
  int32_t lo, hi;
  tail_range(a, j, &lo, &hi);
  if (lo == hi) return;
  const int bt = 3 * a.cut;
  const int32_t t0 = a.bstart[bt], rt = a.brec[bt];
  const int H = a.sheight[rs];
  for (int h = H; h > a.cut; --h) {
    for (int32_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
      if (a.sheight[s] != h) continue;
      const int2 cc = a.sc[s];
      const int64_t rw = rt + (int64_t)(s - t0) * kRecMax;
      T Lp[6];
      load6(a.xs + (int64_t)s * 6, Lp);
      const int type = (cc.x >= 0) + (cc.y >= 0);
      if (type == 0) down_slot<T, 0>(a, s, rw, Lp);
      else if (type == 1) down_slot<T, 1>(a, s, rw, Lp);
      else down_slot<T, 2>(a, s, rw, Lp);
    }
    __syncthreads();
  }
}

template <typename T>
ApplyArgs<T> make_args(const Ctx& c, const T* rec, T* xs, const T* in, T* out) {
  ApplyArgs<T> a;
  a.N = c.N; a.off = c.off; a.perm = c.perm; a.sc = c.sc; a.sroff = c.sroff; a.sheight = c.sheight;
  a.sid = c.sid; a.bstart = c.bstart; a.brec = c.brec; a.root_slot = c.root_slot; a.cut = c.cut;
  a.rec = rec; a.xs = xs; a.in = in; a.out = out;
  return a;
}

template <typename T>
zq_status run_up(Ctx& c, const T* rec, T* xs, const T* v, T* out) {
  ApplyArgs<T> a = make_args<T>(c, rec, xs, v, out);
  const int grid = c.num_sms * 8;
  for (int h = 1; h <= c.cut; ++h) {
    time_begin(c, "up_level");
    k_up_level<T><<<grid, kThreads, 0, c.stream>>>(a, h);
    time_end(c, "up_level");
  }
  time_begin(c, "up_tail");
  k_up_tail<T><<<(unsigned)c.m, kThreads, 0, c.stream>>>(a);
  time_end(c, "up_tail");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

template <typename T>
zq_status run_down(Ctx& c, const T* rec, T* xs, const T* w, T* out) {
  ApplyArgs<T> a = make_args<T>(c, rec, xs, w, out);
  time_begin(c, "down_tail");
  k_down_tail<T><<<(unsigned)c.m, kThreads, 0, c.stream>>>(a);
  time_end(c, "down_tail");
  const int grid = c.num_sms * 8;
  for (int h = c.cut; h >= 1; --h) {
    time_begin(c, "down_level");
    k_down_level<T><<<grid, kThreads, 0, c.stream>>>(a, h);
    time_end(c, "down_level");
  }
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

}  // namespace

zq_status launch_apply_Q(Ctx& c, zq_prec prec, const void* v, int64_t /*ldv*/, void* out) {
  if (prec == ZQ_FP64)
    return run_up<double>(c, c.rec64, c.x64, static_cast<const double*>(v), static_cast<double*>(out));
  return run_up<float>(c, c.rec32, c.x32, static_cast<const float*>(v), static_cast<float*>(out));
}

zq_status launch_apply_QT(Ctx& c, zq_prec prec, const void* w, void* out, int64_t /*ldo*/) {
  if (prec == ZQ_FP64)
    return run_down<double>(c, c.rec64, c.x64, static_cast<const double*>(w), static_cast<double*>(out));
  return run_down<float>(c, c.rec32, c.x32, static_cast<const float*>(w), static_cast<float*>(out));
}

}  // namespace zq
