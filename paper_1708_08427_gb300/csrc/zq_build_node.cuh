// zq_build_node.cuh -- one node transform of Sec. 3, shared by the level
// build (zq_build.cu) and the fused per-body step (zq_fused.cu).
//
// For a node p with children x (lower half) and y (upper half):
//   n = n_x + n_y, centroid c_p = (n_x c_x + n_y c_y) / n (evaluated as
//       c_x - (n_y / n)(c_x - c_y): one FP64 fused multiply-add per axis
//       beside the offset below),
//   alpha = sqrt(n_x / n), beta = sqrt(n_y / n),
//   K = sqrt(n_x n / n_y) R21 with R21 = [c_x - c_p]x, which equals
//       sqrt(n_x n_y / n) [c_x - c_y]x  (c_x - c_p = (n_y / n)(c_x - c_y)),
//   M = [T22_x | T22_y | K] (3 x k; a leaf child has no T22 block, Case II),
//   M = [T22_p 0] G by Householder reflections of A = M^T (Eq. 3.5; LAPACK
//       dgeqrf convention: beta_j = -sign(alpha_j) ||x||, no reflection when
//       the part below the diagonal is exactly zero; then R's diagonal made
//       nonnegative; T22_p = R^T, G = Q^T);
//       before each reflection, a column whose entries (diagonal down) all
//       have binary exponents more than 40 below that of M's largest entry
//       is set to zero (numerical rank decision), so rank-deficient M
//       (collinear or coincident beads) give a transform that does not
//       depend on rounding noise; other columns are reduced as they are.
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
// The node code is written over a real type (zq_real.cuh): native double,
// or double-single pairs of floats evaluated on the FP32 pipes, selected per
// build.  Centroids and the offset d = c_x - c_y are always computed in
// FP64 from FP64 coordinates (cancellation between nearby absolute
// positions needs the full 53 bits); K, T22 and the reflections use the
// chosen type.  A slot's state: centroid (3 doubles), T22 (6 values of the
// chosen type, 8 bytes each).  The state is indexed by the caller's node
// numbering (a slot of the level schedule, or a node id).
#pragma once

#include "zq_internal.cuh"
#include "zq_real.cuh"

namespace zq {

namespace {

struct BuildArgs {
  const double* x;
  const double* y;
  const double* z;
  const int64_t* off;
  const int32_t* perm;  // tree position -> bead (the fused step's leaf lookup)
  const int4* sc;       // per slot: children (x, y, n_x, n_y), see kids_by_id
  const int32_t* cnt;   // bead counts by node id (the fused step's child lookup)
  const uint8_t* sheight;
  const int32_t* sid;
  const int32_t* bstart;
  const int32_t* srw;   // record offset of each slot, 4-word units (uint32)
  const double* ctab;   // sqrt(n) [0, kCountTab), 1/sqrt(n) [kCountTab, 2 kCountTab)
  const float2* ctab2;  // the same as double-single pairs
  int cut;
  void* st;             // kState words of 8 bytes per slot, in the build type
  double* rec64;        // compact records (null: not wanted)
  float* rec32;
  int32_t* err;
};

template <class R>
struct Child {
  int n;
  double c[3];  // centroid
  R L[6];       // packed lower triangle (L00, L10, L11, L20, L21, L22)
};

// A node's children are passed as (x, y, n_x, n_y): x, y >= 0 index a
// child's state, x, y < 0 are leaves given as -1 - the bead's coordinate
// index; n_x, n_y are the children's bead counts.  Every load a node needs
// (state, count table, a leaf's coordinates) depends on these four words
// only, so they issue together.
__device__ __forceinline__ int4 kids_by_id(const BuildArgs& a, int32_t l, int32_t r) {
  return make_int4(l >= 0 ? l : -1 - a.perm[leaf_pos(l)], r >= 0 ? r : -1 - a.perm[leaf_pos(r)],
                   l >= 0 ? a.cnt[l] : 1, r >= 0 ? a.cnt[r] : 1);
}

template <class R>
__device__ __forceinline__ void load_leaf(const BuildArgs& a, int32_t code, Child<R>& ch) {
  const int32_t i = -1 - code;
  ch.n = 1;
  ch.c[0] = a.x[i];
  ch.c[1] = a.y[i];
  ch.c[2] = a.z[i];
}

// A slot's state is 10 words of 8 bytes (80 bytes, 16-byte aligned): the
// centroid, T22's six values in the build type (bit patterns), a pad.  It is
// moved as five 16-byte words.
template <class R>
__device__ __forceinline__ double as_word(R v) {
  static_assert(sizeof(R) == 8, "state words are 8 bytes");
  double d;
  memcpy(&d, &v, 8);
  return d;
}

template <class R>
__device__ __forceinline__ R from_word(double d) {
  R v;
  memcpy(&v, &d, 8);
  return v;
}

template <class R>
__device__ __forceinline__ void load_node(const BuildArgs& a, int32_t slot, int n, Child<R>& ch) {
  const double2* s = reinterpret_cast<const double2*>(reinterpret_cast<const double*>(a.st) + (int64_t)slot * kState);
  ch.n = n;
  double w[10];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const double2 q = s[i];
    w[2 * i] = q.x;
    w[2 * i + 1] = q.y;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) ch.c[i] = w[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) ch.L[i] = from_word<R>(w[3 + i]);
}

template <class R>
struct Geo {
  double cp[3];
  R d[3], al, be, sk;
};

template <class R> __device__ __forceinline__ R table(const BuildArgs& a, int i);
template <> __device__ __forceinline__ double table<double>(const BuildArgs& a, int i) { return __ldg(a.ctab + i); }
template <> __device__ __forceinline__ dd table<dd>(const BuildArgs& a, int i) {
  const float2 v = __ldg(a.ctab2 + i);
  return dd_make(v.x, v.y);
}

template <class R>
__device__ __forceinline__ R count_sqrt(const BuildArgs& a, int n) {
  if (n < kCountTab) return table<R>(a, n);
  return Real<R>::rcp(Real<R>::rsqrt(Real<R>::from_int(n)));
}
template <class R>
__device__ __forceinline__ R count_rsqrt(const BuildArgs& a, int n) {
  if (n < kCountTab) return table<R>(a, kCountTab + n);
  return Real<R>::rsqrt(Real<R>::from_int(n));
}

template <class R>
__device__ __forceinline__ void geometry(const BuildArgs& a, const Child<R>& X, const Child<R>& Y, Geo<R>& g) {
  const R sx = count_sqrt<R>(a, X.n), sy = count_sqrt<R>(a, Y.n), r = count_rsqrt<R>(a, X.n + Y.n);
  const int n = X.n + Y.n;
  const double rd = n < kCountTab ? __ldg(a.ctab + kCountTab + n) : ::rsqrt((double)n);
  const double wy = (double)Y.n * (rd * rd);  // n_y / n
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    // c_p = (n_x c_x + n_y c_y) / n = c_x - (n_y / n) d: the offset d is
    // needed anyway, so the centroid takes one fused multiply-add
    const double d = X.c[i] - Y.c[i];
    g.cp[i] = fma(-wy, d, X.c[i]);
    g.d[i] = Real<R>::from_double(d);
  }
  g.al = sx * r;
  g.be = sy * r;
  g.sk = sx * sy * r;
}

// Case I: n_x = n_y = 1, n = 2.
template <class R>
__device__ __forceinline__ void geometry_pair(const Child<R>& X, const Child<R>& Y, Geo<R>& g) {
  const R root_half = Real<R>::from_double(0.70710678118654757);  // sqrt(1/2), correctly rounded
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double d = X.c[i] - Y.c[i];
    g.cp[i] = fma(-0.5, d, X.c[i]);  // (c_x + c_y) / 2
    g.d[i] = Real<R>::from_double(d);
  }
  g.al = g.be = g.sk = root_half;
}

template <class R, int W>
__device__ __forceinline__ void store(const BuildArgs& a, int64_t slot, int64_t rw, const R (&rec)[W],
                                      const double* cp, const R* L) {
  double2* st = reinterpret_cast<double2*>(reinterpret_cast<double*>(a.st) + slot * kState);
  double w[10];
#pragma unroll
  for (int i = 0; i < 3; ++i) w[i] = cp[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) w[3 + i] = as_word<R>(L[i]);
  w[9] = 0.0;
#pragma unroll
  for (int i = 0; i < 5; ++i) st[i] = make_double2(w[2 * i], w[2 * i + 1]);
  if (a.rec64) {
    double2* r = reinterpret_cast<double2*>(a.rec64 + rw);
#pragma unroll
    for (int i = 0; i < W / 2; ++i)
      r[i] = make_double2(Real<R>::to_double(rec[2 * i]), Real<R>::to_double(rec[2 * i + 1]));
  }
  if (a.rec32) {
    float4* r = reinterpret_cast<float4*>(a.rec32 + rw);
#pragma unroll
    for (int i = 0; i < W / 4; ++i)
      r[i] = make_float4(Real<R>::to_float(rec[4 * i]), Real<R>::to_float(rec[4 * i + 1]),
                         Real<R>::to_float(rec[4 * i + 2]), Real<R>::to_float(rec[4 * i + 3]));
  }
}

// ------------------------------------------------------------ Case I
template <class R>
__device__ void node_case1(const BuildArgs& a, int64_t s, int4 cc, int64_t rw) {
  using RT = Real<R>;
  Child<R> X, Y;
  load_leaf(a, cc.x, X);
  load_leaf(a, cc.y, Y);
  Geo<R> g;
  geometry_pair(X, Y, g);
  const R zero = RT::from_float(0.0f), one = RT::from_float(1.0f);
  R rec[12];
  rec[0] = g.al;
  rec[1] = g.be;
  rec[11] = zero;
  R L[6];
  const R* d = g.d;
  const R dn2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (RT::is_zero(dn2)) {
#pragma unroll
    for (int i = 0; i < 9; ++i) rec[2 + i] = (i % 4 == 0) ? one : zero;
#pragma unroll
    for (int i = 0; i < 6; ++i) L[i] = zero;
    atomicOr(a.err, kErrDegenerate);
  } else {
    const R rdn = RT::rsqrt(dn2), dn = dn2 * rdn;
    const R h[3] = {d[0] * rdn, d[1] * rdn, d[2] * rdn};
    R g1[3];
    if (!RT::is_zero(d[1]) || !RT::is_zero(d[2])) {  // e_x x d, first row of U in Eq. 3.10
      const R rs = RT::rsqrt(d[1] * d[1] + d[2] * d[2]);
      g1[0] = zero; g1[1] = -(d[2] * rs); g1[2] = d[1] * rs;
    } else {                                           // d along x: e_y x d
      g1[0] = zero; g1[1] = zero; g1[2] = RT::ge_zero(d[0]) ? -one : one;
    }
    const R g2[3] = {h[1] * g1[2] - h[2] * g1[1], h[2] * g1[0] - h[0] * g1[2],
                     h[0] * g1[1] - h[1] * g1[0]};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      rec[2 + i] = g1[i];
      rec[5 + i] = g2[i];
      rec[8 + i] = -h[i];
    }
    const R sl = g.sk * dn;  // T22 = sk |d| [g2, -g1, 0]
    L[0] = sl * g2[0];
    L[1] = sl * g2[1];
    L[2] = -(sl * g1[1]);
    L[3] = sl * g2[2];
    L[4] = -(sl * g1[2]);
    L[5] = zero;
  }
  store<R, 12>(a, s, rw, rec, g.cp, L);
}

// Pairwise sum of v[B..E), all of one sign.
template <class R, int B, int E>
__device__ __forceinline__ R sum_same(const R* v) {
  if constexpr (E - B == 1) {
    return v[B];
  } else {
    constexpr int kMid = (B + E) / 2;
    return Real<R>::add_same(sum_same<R, B, kMid>(v), sum_same<R, kMid, E>(v));
  }
}

// One Householder step (LAPACK dlarfg convention) on a column whose
// possibly nonzero entries below the diagonal are x[0..M-1]; al is the
// diagonal entry.  Returns tau (0: no reflection) and scales x into the
// tail of v (v_j = 1 implicit); al becomes beta.
template <class R, int M>
__device__ __forceinline__ R reflector(R& al, R (&x)[M]) {
  using RT = Real<R>;
  // the sums here add terms of one sign (squares; 1 and |al| / norm; al and
  // -be, which has al's sign), so they take the cheaper one-sign sum; the
  // squares in a pairwise tree
  R sq[M];
#pragma unroll
  for (int i = 0; i < M; ++i) sq[i] = RT::sqr(x[i]);
  const R xn2 = sum_same<R, 0, M>(sq);
  if (RT::is_zero(xn2)) {
#pragma unroll
    for (int i = 0; i < M; ++i) x[i] = RT::from_float(0.0f);
    return RT::from_float(0.0f);
  }
  const R n2 = RT::add_same(RT::sqr(al), xn2);
  const R rnorm = RT::rsqrt(n2);
  const R norm = n2 * rnorm;
  const R be = RT::ge_zero(al) ? -norm : norm;
  const R tau = RT::add_same(RT::from_float(1.0f), RT::abs(al) * rnorm);  // = (be - al) / be
  const R rden = RT::rcp(RT::add_same(al, -be));
#pragma unroll
  for (int i = 0; i < M; ++i) x[i] = x[i] * rden;
  al = be;
  return tau;
}

// The numerical rank decision: the column to be reduced (its entries from
// the diagonal down) is set to zero when every entry's exponent is more
// than 40 below M's largest (lim); otherwise it is left as it is.
template <class R, class... Rs>
__device__ __forceinline__ void flush_col(int lim, R& a, Rs&... rest) {
  using RT = Real<R>;
  const bool noise = (RT::bexp(a) < lim) && ((RT::bexp(rest) < lim) && ...);
  if (noise) {
    a = RT::from_float(0.0f);
    ((rest = RT::from_float(0.0f)), ...);
  }
}

// After the three reflections: the rank test, then T22's diagonal made
// nonnegative.  Row j of R (column j of T22) and row j of G change sign
// together; the flip of G's row j is recorded in the sign bit of tau_j
// (tau_j >= 0 otherwise; -0.0 when H_j = I).  A node is flagged degenerate
// when a pivot is zero or more than 33 binary orders below M's largest
// entry (lim + 40): collinear or coincident beads below it.
template <class R>
__device__ __forceinline__ void finish_lq(const BuildArgs& a, int lim, R& A00, R& A01, R& A02, R& A11,
                                          R& A12, R& A22, R* rec) {
  using RT = Real<R>;
  const int lo = lim + 7;
  if (RT::is_zero(A00) || RT::is_zero(A11) || RT::is_zero(A22) || RT::bexp(A00) < lo ||
      RT::bexp(A11) < lo || RT::bexp(A22) < lo)
    atomicOr(a.err, kErrDegenerate);
  if (!RT::ge_zero(A00)) { A00 = -A00; A01 = -A01; A02 = -A02; rec[2] = -rec[2]; }
  if (!RT::ge_zero(A11)) { A11 = -A11; A12 = -A12; rec[3] = -rec[3]; }
  if (!RT::ge_zero(A22)) { A22 = -A22; rec[4] = -rec[4]; }
}

// ------------------------------------------------- k = 6 (Case II)
// A rows: 0-2 = T22_c^T of the internal child, 3-5 = K^T.
template <class R>
__device__ void node_hh6(const BuildArgs& a, int64_t s, int4 cc, int64_t rw) {
  using RT = Real<R>;
  Child<R> X, Y;
  const bool xi = cc.x >= 0;
  if (xi) { load_node(a, cc.x, cc.z, X); load_leaf(a, cc.y, Y); }
  else { load_leaf(a, cc.x, X); load_node(a, cc.y, cc.w, Y); }
  Geo<R> g;
  geometry(a, X, Y, g);
  const R* Lc = xi ? X.L : Y.L;
  const R zero = RT::from_float(0.0f);
  const R kx = g.sk * g.d[0], ky = g.sk * g.d[1], kz = g.sk * g.d[2];
  R A00 = Lc[0], A01 = Lc[1], A02 = Lc[3];
  R A11 = Lc[2], A12 = Lc[4];
  R A22 = Lc[5];
  R A31 = kz, A32 = -ky;
  R A40 = -kz, A41 = zero, A42 = kx;
  R A50 = ky, A51 = -kx, A52 = zero;
  const int lim = max(max(max(RT::bexp(A00), RT::bexp(A01)), max(RT::bexp(A02), RT::bexp(A11))),
                      max(max(RT::bexp(A12), RT::bexp(A22)),
                          max(max(RT::bexp(kx), RT::bexp(ky)), RT::bexp(kz)))) - 40;
  R rec[16];
  rec[0] = g.al;
  rec[1] = g.be;
  rec[13] = rec[14] = rec[15] = zero;
  // H1: column 0, rows 4, 5 below the diagonal
  flush_col(lim, A00, A40, A50);
  {
    R x[2] = {A40, A50};
    const R tau = reflector<R, 2>(A00, x);
    const R v4 = x[0], v5 = x[1];
    R w = (A01 + v5 * A51) * tau;
    A01 -= w; A41 -= w * v4; A51 -= w * v5;
    w = (A02 + v4 * A42) * tau;
    A02 -= w; A42 -= w * v4; A52 -= w * v5;
    rec[2] = tau; rec[5] = v4; rec[6] = v5;
  }
  // H2: column 1, rows 3, 4, 5
  flush_col(lim, A11, A31, A41, A51);
  {
    R x[3] = {A31, A41, A51};
    const R tau = reflector<R, 3>(A11, x);
    const R v3 = x[0], v4 = x[1], v5 = x[2];
    const R w = (A12 + v3 * A32 + v4 * A42 + v5 * A52) * tau;
    A12 -= w; A32 -= w * v3; A42 -= w * v4; A52 -= w * v5;
    rec[3] = tau; rec[7] = v3; rec[8] = v4; rec[9] = v5;
  }
  // H3: column 2, rows 3, 4, 5
  flush_col(lim, A22, A32, A42, A52);
  {
    R x[3] = {A32, A42, A52};
    const R tau = reflector<R, 3>(A22, x);
    rec[4] = tau; rec[10] = x[0]; rec[11] = x[1]; rec[12] = x[2];
  }
  finish_lq(a, lim, A00, A01, A02, A11, A12, A22, rec);
  const R L[6] = {A00, A01, A11, A02, A12, A22};
  store<R, 16>(a, s, rw, rec, g.cp, L);
}

// ------------------------------------------------- k = 9 (general)
// A rows: 0-2 = T22_x^T, 3-5 = T22_y^T, 6-8 = K^T.
template <class R>
__device__ void node_hh9(const BuildArgs& a, int64_t s, int4 cc, int64_t rw) {
  using RT = Real<R>;
  Child<R> X, Y;
  load_node(a, cc.x, cc.z, X);
  load_node(a, cc.y, cc.w, Y);
  Geo<R> g;
  geometry(a, X, Y, g);
  const R zero = RT::from_float(0.0f);
  const R kx = g.sk * g.d[0], ky = g.sk * g.d[1], kz = g.sk * g.d[2];
  R A00 = X.L[0], A01 = X.L[1], A02 = X.L[3];
  R A11 = X.L[2], A12 = X.L[4];
  R A22 = X.L[5];
  R A30 = Y.L[0], A31 = Y.L[1], A32 = Y.L[3];
  R A41 = Y.L[2], A42 = Y.L[4];
  R A52 = Y.L[5];
  R A61 = kz, A62 = -ky;
  R A70 = -kz, A71 = zero, A72 = kx;
  R A80 = ky, A81 = -kx, A82 = zero;
  const int lim = max(max(max(max(RT::bexp(A00), RT::bexp(A01)), max(RT::bexp(A02), RT::bexp(A11))),
                          max(max(RT::bexp(A12), RT::bexp(A22)), max(RT::bexp(A30), RT::bexp(A31)))),
                      max(max(max(RT::bexp(A32), RT::bexp(A41)), max(RT::bexp(A42), RT::bexp(A52))),
                          max(max(RT::bexp(kx), RT::bexp(ky)), RT::bexp(kz)))) - 40;
  R rec[20];
  rec[0] = g.al;
  rec[1] = g.be;
  rec[19] = zero;
  // H1: column 0, rows 3, 7, 8
  flush_col(lim, A00, A30, A70, A80);
  {
    R x[3] = {A30, A70, A80};
    const R tau = reflector<R, 3>(A00, x);
    const R v3 = x[0], v7 = x[1], v8 = x[2];
    R w = (A01 + v3 * A31 + v8 * A81) * tau;
    A01 -= w; A31 -= w * v3; A71 -= w * v7; A81 -= w * v8;
    w = (A02 + v3 * A32 + v7 * A72) * tau;
    A02 -= w; A32 -= w * v3; A72 -= w * v7; A82 -= w * v8;
    rec[2] = tau; rec[5] = v3; rec[6] = v7; rec[7] = v8;
  }
  // H2: column 1, rows 3, 4, 6, 7, 8
  flush_col(lim, A11, A31, A41, A61, A71, A81);
  {
    R x[5] = {A31, A41, A61, A71, A81};
    const R tau = reflector<R, 5>(A11, x);
    const R v3 = x[0], v4 = x[1], v6 = x[2], v7 = x[3], v8 = x[4];
    const R w = (A12 + v3 * A32 + v4 * A42 + v6 * A62 + v7 * A72 + v8 * A82) * tau;
    A12 -= w; A32 -= w * v3; A42 -= w * v4; A62 -= w * v6; A72 -= w * v7; A82 -= w * v8;
    rec[3] = tau; rec[8] = v3; rec[9] = v4; rec[10] = v6; rec[11] = v7; rec[12] = v8;
  }
  // H3: column 2, rows 3..8
  flush_col(lim, A22, A32, A42, A52, A62, A72, A82);
  {
    R x[6] = {A32, A42, A52, A62, A72, A82};
    const R tau = reflector<R, 6>(A22, x);
    rec[4] = tau;
#pragma unroll
    for (int i = 0; i < 6; ++i) rec[13 + i] = x[i];
  }
  finish_lq(a, lim, A00, A01, A02, A11, A12, A22, rec);
  const R L[6] = {A00, A01, A11, A02, A12, A22};
  store<R, 20>(a, s, rw, rec, g.cp, L);
}

template <class R>
__device__ __forceinline__ void build_slot(const BuildArgs& a, int64_t s, int type, int64_t rw) {
  const int4 cc = a.sc[s];
  if (type == 0) node_case1<R>(a, s, cc, rw);
  else if (type == 1) node_hh6<R>(a, s, cc, rw);
  else node_hh9<R>(a, s, cc, rw);
}

}  // namespace

}  // namespace zq
