// zq_build.cu -- per-node transforms of Sec. 3 in FP64.
//
// For a node p with children x (lower half) and y (upper half):
//   n = n_x + n_y, centroid c_p = (n_x c_x + n_y c_y) / n,
//   alpha = sqrt(n_x / n), beta = sqrt(n_y / n),
//   K = sqrt(n_x n / n_y) R21 with R21 = [c_x - c_p]x, which equals
//       sqrt(n_x n_y / n) [c_x - c_y]x  (c_x - c_p = (n_y / n)(c_x - c_y)),
//   M = [T22_x | T22_y | K] (3 x k; a leaf child has no T22 block, Case II),
//   M = [T22_p 0] G by Householder reflections of A = M^T (Eq. 3.5; LAPACK
//       dgeqrf convention: beta_j = -sign(alpha_j) ||x||, no reflection when
//       the part below the diagonal is exactly zero; T22_p = R^T, G = Q^T);
//       before each reflection, column entries whose binary exponent is
//       more than 40 below that of M's largest entry are set to zero, so
//       rank-deficient M (collinear or coincident beads) give a transform
//       that does not depend on rounding noise.
// Case I (two leaves, Eqs. 3.9-3.10): G rows g1 = (e_x x d)/|e_x x d|
// (e_y x d when d has no y, z part), g2 = dhat x g1, g3 = -dhat, and
// T22_p = sqrt(n_x n_y / n) |d| [g2, -g1, 0]; d = 0 gives G = I, T22 = 0
// and the degenerate warning.
//
// A has structural zeros (T22 blocks are lower triangular, [d]x has a zero
// diagonal); the reflections below touch only the entries that can be
// nonzero, which is exact (the skipped products are by exact zeros).
//
// FP64 runs at 1/64 of the FP32 rate on this GPU and square roots and
// divisions expand to long instruction sequences, so: sqrt(n) and
// 1/sqrt(n) of bead counts come from a table, Case I (n_x = n_y = 1) uses
// the constants sqrt(1/2) and 1/2, each reflection takes one reciprocal
// square root and one division, and the zero test works on exponent bits.
//
// Schedule: heights 1..cut level by level over all bodies (one launch per
// height, nodes sorted by type inside a height), then the remaining nodes
// one thread block per body.  A node's children are finished before it.
#include "zq_internal.cuh"

namespace zq {

namespace {

constexpr int kThreads = 256;

struct BuildArgs {
  const double* x;
  const double* y;
  const double* z;
  const int64_t* off;
  const int32_t* perm;
  const int2* sc;
  const int32_t* scnt;
  const uint8_t* sheight;
  const int32_t* sid;
  const int32_t* bstart;
  const int32_t* brec;
  const int32_t* root_slot;
  const double* ctab;  // sqrt(n) [0, kCountTab), 1/sqrt(n) [kCountTab, 2 kCountTab)
  int cut;
  double* st64;
  double* rec64;  // compact records (may be null: not wanted)
  float* rec32;
  int32_t* err;
};

struct Child {
  int n;
  double c[3];
  double L[6];  // packed lower triangle (L00, L10, L11, L20, L21, L22)
};

__device__ __forceinline__ void load_leaf(const BuildArgs& a, int32_t code, Child& ch) {
  const int32_t i = a.perm[leaf_pos(code)];
  ch.n = 1;
  ch.c[0] = a.x[i];
  ch.c[1] = a.y[i];
  ch.c[2] = a.z[i];
}

__device__ __forceinline__ void load_node(const BuildArgs& a, int32_t slot, Child& ch) {
  const double2* s = reinterpret_cast<const double2*>(a.st64 + (int64_t)slot * kState);
  const double2 s0 = s[0], s1 = s[1], s2 = s[2], s3 = s[3], s4 = s[4];
  ch.n = a.scnt[slot];
  ch.c[0] = s0.x; ch.c[1] = s0.y; ch.c[2] = s1.x;
  ch.L[0] = s1.y; ch.L[1] = s2.x; ch.L[2] = s2.y; ch.L[3] = s3.x; ch.L[4] = s3.y; ch.L[5] = s4.x;
}

struct Geo {
  double cp[3], d[3], al, be, sk;
};

__device__ __forceinline__ double count_sqrt(const BuildArgs& a, int n) {
  return n < kCountTab ? __ldg(a.ctab + n) : sqrt((double)n);
}
__device__ __forceinline__ double count_rsqrt(const BuildArgs& a, int n) {
  return n < kCountTab ? __ldg(a.ctab + kCountTab + n) : rsqrt((double)n);
}

__device__ __forceinline__ void geometry(const BuildArgs& a, const Child& X, const Child& Y, Geo& g) {
  const double sx = count_sqrt(a, X.n), sy = count_sqrt(a, Y.n), r = count_rsqrt(a, X.n + Y.n);
  const double rn = r * r, nx = (double)X.n, ny = (double)Y.n;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    g.cp[i] = (nx * X.c[i] + ny * Y.c[i]) * rn;
    g.d[i] = X.c[i] - Y.c[i];
  }
  g.al = sx * r;
  g.be = sy * r;
  g.sk = sx * sy * r;
}

// Case I: n_x = n_y = 1, n = 2.
__device__ __forceinline__ void geometry_pair(const Child& X, const Child& Y, Geo& g) {
  constexpr double kRootHalf = 0.70710678118654757;  // sqrt(1/2), correctly rounded
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    g.cp[i] = (X.c[i] + Y.c[i]) * 0.5;
    g.d[i] = X.c[i] - Y.c[i];
  }
  g.al = g.be = g.sk = kRootHalf;
}

// Biased binary exponent of a double (0 for zero and subnormals).
__device__ __forceinline__ int bexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

template <int W>
__device__ __forceinline__ void store(const BuildArgs& a, int64_t slot, int64_t rw, const double (&rec)[W],
                                      const double* cp, const double* L) {
  double2* st = reinterpret_cast<double2*>(a.st64 + slot * kState);
  st[0] = make_double2(cp[0], cp[1]);
  st[1] = make_double2(cp[2], L[0]);
  st[2] = make_double2(L[1], L[2]);
  st[3] = make_double2(L[3], L[4]);
  st[4] = make_double2(L[5], 0.0);
  if (a.rec64) {
    double2* r = reinterpret_cast<double2*>(a.rec64 + rw);
#pragma unroll
    for (int i = 0; i < W / 2; ++i) r[i] = make_double2(rec[2 * i], rec[2 * i + 1]);
  }
  if (a.rec32) {
    float4* r = reinterpret_cast<float4*>(a.rec32 + rw);
#pragma unroll
    for (int i = 0; i < W / 4; ++i)
      r[i] = make_float4((float)rec[4 * i], (float)rec[4 * i + 1], (float)rec[4 * i + 2], (float)rec[4 * i + 3]);
  }
}

// ------------------------------------------------------------ Case I
__device__ void node_case1(const BuildArgs& a, int64_t s, int2 cc, int64_t rw) {
  Child X, Y;
  load_leaf(a, cc.x, X);
  load_leaf(a, cc.y, Y);
  Geo g;
  geometry_pair(X, Y, g);
  double rec[12];
  rec[0] = g.al;
  rec[1] = g.be;
  rec[11] = 0.0;
  double L[6];
  const double* d = g.d;
  const double dn2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (dn2 == 0.0) {
#pragma unroll
    for (int i = 0; i < 9; ++i) rec[2 + i] = (i % 4 == 0) ? 1.0 : 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) L[i] = 0.0;
    atomicOr(a.err, kErrDegenerate);
  } else {
    const double rdn = rsqrt(dn2), dn = dn2 * rdn;
    const double h[3] = {d[0] * rdn, d[1] * rdn, d[2] * rdn};
    double g1[3];
    if (d[1] != 0.0 || d[2] != 0.0) {  // e_x x d, first row of U in Eq. 3.10
      const double rs = rsqrt(d[1] * d[1] + d[2] * d[2]);
      g1[0] = 0.0; g1[1] = -d[2] * rs; g1[2] = d[1] * rs;
    } else {                            // d along x: e_y x d
      g1[0] = 0.0; g1[1] = 0.0; g1[2] = d[0] > 0.0 ? -1.0 : 1.0;
    }
    const double g2[3] = {h[1] * g1[2] - h[2] * g1[1], h[2] * g1[0] - h[0] * g1[2],
                          h[0] * g1[1] - h[1] * g1[0]};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      rec[2 + i] = g1[i];
      rec[5 + i] = g2[i];
      rec[8 + i] = -h[i];
    }
    const double sl = g.sk * dn;  // T22 = sk |d| [g2, -g1, 0]
    L[0] = sl * g2[0];
    L[1] = sl * g2[1];
    L[2] = -sl * g1[1];
    L[3] = sl * g2[2];
    L[4] = -sl * g1[2];
    L[5] = 0.0;
  }
  store<12>(a, s, rw, rec, g.cp, L);
}

// One Householder step (LAPACK dlarfg convention) on a column whose
// possibly nonzero entries below the diagonal are x[0..M-1]; al is the
// diagonal entry.  Returns tau (0: no reflection) and scales x into the
// tail of v (v_j = 1 implicit); al becomes beta.
template <int M>
__device__ __forceinline__ double reflector(double& al, double (&x)[M]) {
  double xn2 = 0.0;
#pragma unroll
  for (int i = 0; i < M; ++i) xn2 += x[i] * x[i];
  if (xn2 == 0.0) {
#pragma unroll
    for (int i = 0; i < M; ++i) x[i] = 0.0;
    return 0.0;
  }
  const double n2 = al * al + xn2;
  const double rnorm = rsqrt(n2);
  const double norm = n2 * rnorm;
  const double be = (al >= 0.0) ? -norm : norm;
  const double tau = 1.0 + fabs(al) * rnorm;  // = (be - al) / be
  const double rden = 1.0 / (al - be);
#pragma unroll
  for (int i = 0; i < M; ++i) x[i] *= rden;
  al = be;
  return tau;
}

// The zero rule: entries whose exponent is more than 40 below the largest.
__device__ __forceinline__ void flush(double& v, int lim) {
  if (bexp(v) < lim) v = 0.0;
}

// ------------------------------------------------- k = 6 (Case II)
// A rows: 0-2 = T22_c^T of the internal child, 3-5 = K^T.
__device__ void node_hh6(const BuildArgs& a, int64_t s, int2 cc, int64_t rw) {
  Child X, Y;
  const bool xi = cc.x >= 0;
  if (xi) { load_node(a, cc.x, X); load_leaf(a, cc.y, Y); }
  else { load_leaf(a, cc.x, X); load_node(a, cc.y, Y); }
  Geo g;
  geometry(a, X, Y, g);
  const double* Lc = xi ? X.L : Y.L;
  const double kx = g.sk * g.d[0], ky = g.sk * g.d[1], kz = g.sk * g.d[2];
  // columns of A: a0 (rows 0, 4, 5), a1 (rows 0, 1, 3, 5 + fill 4), a2 (rows 0-4 + fill 5)
  double A00 = Lc[0], A01 = Lc[1], A02 = Lc[3];
  double A11 = Lc[2], A12 = Lc[4];
  double A22 = Lc[5];
  double A31 = kz, A32 = -ky;
  double A40 = -kz, A41 = 0.0, A42 = kx;
  double A50 = ky, A51 = -kx, A52 = 0.0;
  const int tiny = max(max(max(bexp(A00), bexp(A01)), max(bexp(A02), bexp(A11))),
                       max(max(bexp(A12), bexp(A22)), max(max(bexp(kx), bexp(ky)), bexp(kz)))) - 40;
  double rec[16];
  rec[0] = g.al;
  rec[1] = g.be;
  rec[13] = rec[14] = rec[15] = 0.0;
  // H1: column 0, rows 4, 5 below the diagonal
  flush(A00, tiny); flush(A40, tiny); flush(A50, tiny);
  {
    double x[2] = {A40, A50};
    const double tau = reflector<2>(A00, x);
    const double v4 = x[0], v5 = x[1];
    double w = (A01 + v5 * A51) * tau;
    A01 -= w; A41 -= w * v4; A51 -= w * v5;
    w = (A02 + v4 * A42) * tau;
    A02 -= w; A42 -= w * v4; A52 -= w * v5;
    rec[2] = tau; rec[5] = v4; rec[6] = v5;
  }
  // H2: column 1, rows 3, 4, 5
  flush(A11, tiny); flush(A31, tiny); flush(A41, tiny); flush(A51, tiny);
  {
    double x[3] = {A31, A41, A51};
    const double tau = reflector<3>(A11, x);
    const double v3 = x[0], v4 = x[1], v5 = x[2];
    const double w = (A12 + v3 * A32 + v4 * A42 + v5 * A52) * tau;
    A12 -= w; A32 -= w * v3; A42 -= w * v4; A52 -= w * v5;
    rec[3] = tau; rec[7] = v3; rec[8] = v4; rec[9] = v5;
  }
  // H3: column 2, rows 3, 4, 5
  flush(A22, tiny); flush(A32, tiny); flush(A42, tiny); flush(A52, tiny);
  {
    double x[3] = {A32, A42, A52};
    const double tau = reflector<3>(A22, x);
    rec[4] = tau; rec[10] = x[0]; rec[11] = x[1]; rec[12] = x[2];
  }
  const double L[6] = {A00, A01, A11, A02, A12, A22};
  store<16>(a, s, rw, rec, g.cp, L);
}

// ------------------------------------------------- k = 9 (general)
// A rows: 0-2 = T22_x^T, 3-5 = T22_y^T, 6-8 = K^T.
__device__ void node_hh9(const BuildArgs& a, int64_t s, int2 cc, int64_t rw) {
  Child X, Y;
  load_node(a, cc.x, X);
  load_node(a, cc.y, Y);
  Geo g;
  geometry(a, X, Y, g);
  const double kx = g.sk * g.d[0], ky = g.sk * g.d[1], kz = g.sk * g.d[2];
  double A00 = X.L[0], A01 = X.L[1], A02 = X.L[3];
  double A11 = X.L[2], A12 = X.L[4];
  double A22 = X.L[5];
  double A30 = Y.L[0], A31 = Y.L[1], A32 = Y.L[3];
  double A41 = Y.L[2], A42 = Y.L[4];
  double A52 = Y.L[5];
  double A61 = kz, A62 = -ky;
  double A70 = -kz, A71 = 0.0, A72 = kx;
  double A80 = ky, A81 = -kx, A82 = 0.0;
  const int tiny = max(max(max(max(bexp(A00), bexp(A01)), max(bexp(A02), bexp(A11))),
                           max(max(bexp(A12), bexp(A22)), max(bexp(A30), bexp(A31)))),
                       max(max(max(bexp(A32), bexp(A41)), max(bexp(A42), bexp(A52))),
                           max(max(bexp(kx), bexp(ky)), bexp(kz)))) - 40;
  double rec[20];
  rec[0] = g.al;
  rec[1] = g.be;
  rec[19] = 0.0;
  // H1: column 0, rows 3, 7, 8
  flush(A00, tiny); flush(A30, tiny); flush(A70, tiny); flush(A80, tiny);
  {
    double x[3] = {A30, A70, A80};
    const double tau = reflector<3>(A00, x);
    const double v3 = x[0], v7 = x[1], v8 = x[2];
    double w = (A01 + v3 * A31 + v8 * A81) * tau;
    A01 -= w; A31 -= w * v3; A71 -= w * v7; A81 -= w * v8;
    w = (A02 + v3 * A32 + v7 * A72) * tau;
    A02 -= w; A32 -= w * v3; A72 -= w * v7; A82 -= w * v8;
    rec[2] = tau; rec[5] = v3; rec[6] = v7; rec[7] = v8;
  }
  // H2: column 1, rows 3, 4, 6, 7, 8
  flush(A11, tiny); flush(A31, tiny); flush(A41, tiny); flush(A61, tiny); flush(A71, tiny); flush(A81, tiny);
  {
    double x[5] = {A31, A41, A61, A71, A81};
    const double tau = reflector<5>(A11, x);
    const double v3 = x[0], v4 = x[1], v6 = x[2], v7 = x[3], v8 = x[4];
    const double w = (A12 + v3 * A32 + v4 * A42 + v6 * A62 + v7 * A72 + v8 * A82) * tau;
    A12 -= w; A32 -= w * v3; A42 -= w * v4; A62 -= w * v6; A72 -= w * v7; A82 -= w * v8;
    rec[3] = tau; rec[8] = v3; rec[9] = v4; rec[10] = v6; rec[11] = v7; rec[12] = v8;
  }
  // H3: column 2, rows 3..8
  flush(A22, tiny); flush(A32, tiny); flush(A42, tiny); flush(A52, tiny); flush(A62, tiny);
  flush(A72, tiny); flush(A82, tiny);
  {
    double x[6] = {A32, A42, A52, A62, A72, A82};
    const double tau = reflector<6>(A22, x);
    rec[4] = tau;
#pragma unroll
    for (int i = 0; i < 6; ++i) rec[13 + i] = x[i];
  }
  const double L[6] = {A00, A01, A11, A02, A12, A22};
  store<20>(a, s, rw, rec, g.cp, L);
}

__device__ __forceinline__ void build_slot(const BuildArgs& a, int64_t s, int type, int64_t rw) {
  const int2 cc = a.sc[s];
  if (type == 0) node_case1(a, s, cc, rw);
  else if (type == 1) node_hh6(a, s, cc, rw);
  else node_hh9(a, s, cc, rw);
}

__global__ void __launch_bounds__(kThreads) k_build_level(BuildArgs a, int h) {
  const int b0 = 3 * (h - 1);
  const int32_t s0 = a.bstart[b0], s1 = a.bstart[b0 + 1], s2 = a.bstart[b0 + 2], s3 = a.bstart[b0 + 3];
  const int32_t r0 = a.brec[b0], r1 = a.brec[b0 + 1], r2 = a.brec[b0 + 2];
  for (int64_t s = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < s3;
       s += (int64_t)gridDim.x * blockDim.x) {
    if (s < s1) build_slot(a, s, 0, r0 + (s - s0) * rec_words(0));
    else if (s < s2) build_slot(a, s, 1, r1 + (s - s1) * rec_words(1));
    else build_slot(a, s, 2, r2 + (s - s2) * rec_words(2));
  }
}

// Nodes above the cut: one block per body, height by height.
__global__ void __launch_bounds__(kThreads) k_build_tail(BuildArgs a) {
  const int32_t j = blockIdx.x;
  const int bt = 3 * a.cut;
  const int32_t t0 = a.bstart[bt], t1 = a.bstart[bt + 1];
  int32_t lo, hi;
  id_range(a.sid, t0, t1, a.off[j] - j, a.off[j + 1] - (j + 1), &lo, &hi);
  if (lo == hi) return;
  const int H = a.sheight[a.root_slot[j]];
  const int32_t rt = a.brec[bt];
  for (int h = a.cut + 1; h <= H; ++h) {
    for (int32_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
      if (a.sheight[s] != h) continue;
      const int2 cc = a.sc[s];
      build_slot(a, s, (cc.x >= 0) + (cc.y >= 0), rt + (int64_t)(s - t0) * kRecMax);
    }
    __syncthreads();
  }
}

}  // namespace

zq_status launch_build(Ctx& c, const double* x, const double* y, const double* z, int which) {
  BuildArgs a;
  a.x = x; a.y = y; a.z = z;
  a.off = c.off; a.perm = c.perm; a.sc = c.sc; a.scnt = c.scnt; a.sheight = c.sheight; a.sid = c.sid;
  a.bstart = c.bstart; a.brec = c.brec; a.root_slot = c.root_slot; a.cut = c.cut;
  a.ctab = c.count_tab;
  a.st64 = c.st64;
  a.rec64 = (which & 1) ? c.rec64 : nullptr;
  a.rec32 = (which & 2) ? c.rec32 : nullptr;
  a.err = c.counters + 2;
  const int grid = c.num_sms * 4;
  for (int h = 1; h <= c.cut; ++h) {
    time_begin(c, "build_level");
    k_build_level<<<grid, kThreads, 0, c.stream>>>(a, h);
    time_end(c, "build_level");
  }
  time_begin(c, "build_tail");
  k_build_tail<<<(unsigned)c.m, kThreads, 0, c.stream>>>(a);
  time_end(c, "build_tail");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

}  // namespace zq
