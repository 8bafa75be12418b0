// zq_build.cu -- per-node transforms of Sec. 3 in FP64.
//
// For a node p with children x (lower half) and y (upper half):
//   n = n_x + n_y, centroid c_p = (n_x c_x + n_y c_y) / n,
//   alpha = sqrt(n_x / n), beta = sqrt(n_y / n),
//   K = sqrt(n_x n / n_y) R21 with R21 = [c_x - c_p]x, which equals
//       sqrt(n_x n_y / n) [c_x - c_y]x  (c_x - c_p = (n_y / n)(c_x - c_y)),
//   M = [T22_x | T22_y | K] (3 x k; a leaf child has no T22 block, Case II),
//   M = [T22_p 0] G by Householder reflections of M^T (Eq. 3.5; LAPACK
//       dgeqrf convention: beta_j = -sign(alpha_j) ||x||, no reflection when
//       the part below the diagonal is exactly zero; T22_p = R^T, G = Q^T);
//       before each reflection, column entries <= 2^-44 ||M||_F are set to
//       zero, so rank-deficient M (collinear or coincident beads) give a
//       transform that does not depend on rounding noise.
// Case I (two leaves, Eqs. 3.9-3.10): G rows g1 = (e_x x d)/|e_x x d|
// (e_y x d when d has no y, z part), g2 = dhat x g1, g3 = -dhat, and
// T22_p = sqrt(n_x n_y / n) |d| [g2, -g1, 0]; d = 0 gives G = I, T22 = 0
// and the degenerate warning.
//
// Nodes are processed tile by tile (a tile = subtree of at most `tile`
// beads, one thread block) and inside a tile level by level (heights
// 1, 2, ...); the nodes above the tiles are then processed per body.
// The children's state (centroid, T22) is read from global memory.
#include "zq_internal.cuh"

namespace zq {

namespace {

constexpr int kThreads = 256;

struct BuildArgs {
  const double* x;
  const double* y;
  const double* z;
  const int64_t* off;
  int64_t m;
  const int32_t* perm;
  const int32_t* cl;
  const int32_t* cr;
  const int32_t* cnt;
  const int32_t* first;
  const uint8_t* height;
  const int32_t* tiles;
  const int32_t* top;
  const int32_t* counters;
  const int32_t* top_bodies;
  const int32_t* root;
  double* st64;
  double* rec64;
  float* rec32;
  int32_t* err;
};

struct Child {
  int n;
  double c[3];
  double L[6];  // packed lower triangle, valid for internal children
  bool internal;
};

__device__ inline void load_child(const BuildArgs& a, int32_t code, Child& ch) {
  if (is_leaf(code)) {
    const int32_t i = a.perm[leaf_pos(code)];
    ch.n = 1;
    ch.c[0] = a.x[i];
    ch.c[1] = a.y[i];
    ch.c[2] = a.z[i];
    ch.internal = false;
  } else {
    const double* s = a.st64 + (int64_t)code * kState;
    ch.n = a.cnt[code];
#pragma unroll
    for (int i = 0; i < 3; ++i) ch.c[i] = s[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) ch.L[i] = s[3 + i];
    ch.internal = true;
  }
}

__device__ void build_node(const BuildArgs& a, int64_t q) {
  const int32_t lc = a.cl[q], rc = a.cr[q];
  Child X, Y;
  load_child(a, lc, X);
  load_child(a, rc, Y);
  const double nx = (double)X.n, ny = (double)Y.n, n = nx + ny;
  double cp[3], d[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cp[i] = (nx * X.c[i] + ny * Y.c[i]) / n;
    d[i] = X.c[i] - Y.c[i];
  }
  const double sk = sqrt(nx * ny / n);
  double rec[kRec];
#pragma unroll
  for (int i = 0; i < kRec; ++i) rec[i] = 0.0;
  rec[0] = sqrt(nx / n);
  rec[1] = sqrt(ny / n);
  double Lp[6];

  if (!X.internal && !Y.internal) {
    // Case I, bead & bead (Eqs. 3.9-3.10)
    const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (dn == 0.0) {
      rec[5] = 1.0; rec[9] = 1.0; rec[13] = 1.0;
#pragma unroll
      for (int i = 0; i < 6; ++i) Lp[i] = 0.0;
      atomicOr(a.err, kErrDegenerate);
    } else {
      const double h[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
      double g1[3];
      if (d[1] != 0.0 || d[2] != 0.0) {
        const double s = sqrt(d[1] * d[1] + d[2] * d[2]);
        g1[0] = 0.0; g1[1] = -d[2] / s; g1[2] = d[1] / s;
      } else {
        g1[0] = 0.0; g1[1] = 0.0; g1[2] = -d[0] / fabs(d[0]);
      }
      const double g2[3] = {h[1] * g1[2] - h[2] * g1[1], h[2] * g1[0] - h[0] * g1[2],
                            h[0] * g1[1] - h[1] * g1[0]};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        rec[5 + i] = g1[i];
        rec[8 + i] = g2[i];
        rec[11 + i] = -h[i];
      }
      const double s = sk * dn;
      Lp[0] = s * g2[0];
      Lp[1] = s * g2[1];
      Lp[2] = -s * g1[1];
      Lp[3] = s * g2[2];
      Lp[4] = -s * g1[2];
      Lp[5] = 0.0;
    }
  } else {
    // General node / Case II: Householder QR of A = M^T (k x 3)
    double A[9][3];
    int k = 0;
    if (X.internal) {
      A[0][0] = X.L[0]; A[0][1] = X.L[1]; A[0][2] = X.L[3];
      A[1][0] = 0.0;    A[1][1] = X.L[2]; A[1][2] = X.L[4];
      A[2][0] = 0.0;    A[2][1] = 0.0;    A[2][2] = X.L[5];
      k = 3;
    }
    if (Y.internal) {
      A[k][0] = Y.L[0];   A[k][1] = Y.L[1];   A[k][2] = Y.L[3];
      A[k + 1][0] = 0.0;  A[k + 1][1] = Y.L[2]; A[k + 1][2] = Y.L[4];
      A[k + 2][0] = 0.0;  A[k + 2][1] = 0.0;  A[k + 2][2] = Y.L[5];
      k += 3;
    }
    A[k][0] = sk * 0.0;        A[k][1] = sk * d[2];       A[k][2] = sk * (-d[1]);
    A[k + 1][0] = sk * (-d[2]); A[k + 1][1] = sk * 0.0;    A[k + 1][2] = sk * d[0];
    A[k + 2][0] = sk * d[1];   A[k + 2][1] = sk * (-d[0]); A[k + 2][2] = sk * 0.0;
    k += 3;
    // entries <= 2^-44 ||M||_F are rounding noise of an exact zero
    // (rank-deficient M); they are zeroed before each reflection
    double mn2 = 0.0;
    for (int i = 0; i < k; ++i)
#pragma unroll
      for (int c = 0; c < 3; ++c) mn2 += A[i][c] * A[i][c];
    const double tiny = sqrt(mn2) * 0x1p-44;
    int tail = 5;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      for (int i = j; i < k; ++i)
        if (fabs(A[i][j]) <= tiny) A[i][j] = 0.0;
      double xn2 = 0.0;
      for (int i = j + 1; i < k; ++i) xn2 += A[i][j] * A[i][j];
      if (xn2 != 0.0) {
        const double al = A[j][j];
        const double norm = sqrt(al * al + xn2);
        const double be = (al >= 0.0) ? -norm : norm;
        const double tau = (be - al) / be;
        const double den = al - be;
        double v[9];
        for (int i = j + 1; i < k; ++i) v[i] = A[i][j] / den;
        A[j][j] = be;
        for (int i = j + 1; i < k; ++i) A[i][j] = 0.0;
#pragma unroll
        for (int c = j + 1; c < 3; ++c) {
          double w = A[j][c];
          for (int i = j + 1; i < k; ++i) w += v[i] * A[i][c];
          A[j][c] -= tau * w;
          for (int i = j + 1; i < k; ++i) A[i][c] -= tau * w * v[i];
        }
        rec[2 + j] = tau;
        for (int i = j + 1; i < k; ++i) rec[tail + (i - j - 1)] = v[i];
      }
      tail += k - 1 - j;
    }
    Lp[0] = A[0][0];
    Lp[1] = A[0][1];
    Lp[2] = A[1][1];
    Lp[3] = A[0][2];
    Lp[4] = A[1][2];
    Lp[5] = A[2][2];
  }
  double* st = a.st64 + q * kState;
#pragma unroll
  for (int i = 0; i < 3; ++i) st[i] = cp[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) st[3 + i] = Lp[i];
  double2* r64 = reinterpret_cast<double2*>(a.rec64 + q * kRec);
  float4* r32 = reinterpret_cast<float4*>(a.rec32 + q * kRec);
#pragma unroll
  for (int i = 0; i < kRec / 2; ++i) r64[i] = make_double2(rec[2 * i], rec[2 * i + 1]);
#pragma unroll
  for (int i = 0; i < kRec / 4; ++i)
    r32[i] = make_float4((float)rec[4 * i], (float)rec[4 * i + 1], (float)rec[4 * i + 2],
                         (float)rec[4 * i + 3]);
}

// Per-tile level lists in shared memory: list[lstart[h] .. lstart[h+1]) =
// local indices of the tile's nodes of height h.  Returns the tile height.
__device__ int make_levels(const uint8_t* __restrict__ hgt, int nn, uint16_t* list, int* lstart,
                           int* lcnt, int* hmax) {
  for (int i = threadIdx.x; i < kMaxHeight + 2; i += blockDim.x) lcnt[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < nn; i += blockDim.x) atomicAdd(&lcnt[hgt[i]], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0, H = 0;
    for (int h = 0; h <= kMaxHeight; ++h) {
      lstart[h] = s;
      s += lcnt[h];
      if (lcnt[h]) H = h;
      lcnt[h] = 0;
    }
    lstart[kMaxHeight + 1] = s;
    *hmax = H;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int h = hgt[i];
    list[lstart[h] + atomicAdd(&lcnt[h], 1)] = (uint16_t)i;
  }
  __syncthreads();
  return *hmax;
}

__global__ void __launch_bounds__(kThreads) k_build_tiles(BuildArgs a) {
  extern __shared__ unsigned char smem[];
  __shared__ int lstart[kMaxHeight + 2], lcnt[kMaxHeight + 2], hmax;
  uint16_t* list = reinterpret_cast<uint16_t*>(smem);
  const int ntiles = a.counters[0];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int32_t R = a.tiles[t];
    const int32_t j = body_of_node(a.off, a.m, R);
    const int64_t base = (int64_t)a.first[R] - j;
    const int nn = a.cnt[R] - 1;
    const int H = make_levels(a.height + base, nn, list, lstart, lcnt, &hmax);
    for (int h = 1; h <= H; ++h) {
      for (int p = lstart[h] + threadIdx.x; p < lstart[h + 1]; p += blockDim.x)
        build_node(a, base + list[p]);
      __syncthreads();
    }
  }
}

// Range [lo, hi) of the sorted top-node list holding ids in [a, b).
__device__ inline void top_range(const int32_t* top, int ntop, int64_t a, int64_t b, int* lo,
                                 int* hi) {
  int l = 0, r = ntop;
  while (l < r) { int md = (l + r) >> 1; if (top[md] < a) l = md + 1; else r = md; }
  *lo = l;
  r = ntop;
  while (l < r) { int md = (l + r) >> 1; if (top[md] < b) l = md + 1; else r = md; }
  *hi = l;
}

__global__ void __launch_bounds__(kThreads) k_build_top(BuildArgs a) {
  const int32_t j = a.top_bodies[blockIdx.x];
  const int64_t nb = a.off[j] - j, ne = a.off[j + 1] - (j + 1);
  int lo, hi;
  top_range(a.top, a.counters[1], nb, ne, &lo, &hi);
  const int H = a.height[a.root[j]];
  for (int h = 1; h <= H; ++h) {
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
      const int32_t q = a.top[p];
      if (a.height[q] == h) build_node(a, q);
    }
    __syncthreads();
  }
}

}  // namespace

zq_status launch_build(Ctx& c, const double* x, const double* y, const double* z) {
  BuildArgs a;
  a.x = x; a.y = y; a.z = z;
  a.off = c.off; a.m = c.m;
  a.perm = c.perm; a.cl = c.cl; a.cr = c.cr; a.cnt = c.cnt; a.first = c.first;
  a.height = c.height; a.tiles = c.tiles; a.top = c.top; a.counters = c.counters;
  a.top_bodies = c.top_d; a.root = c.root;
  a.st64 = c.st64; a.rec64 = c.rec64; a.rec32 = c.rec32; a.err = c.counters + 2;
  const size_t smem = (size_t)c.tile * sizeof(uint16_t);
  const int grid = c.num_sms * 8;
  time_begin(c, "build_tiles");
  k_build_tiles<<<grid, kThreads, smem, c.stream>>>(a);
  time_end(c, "build_tiles");
  ZQ_CUDA_TRY(cudaGetLastError());
  if (!c.top_bodies.empty()) {
    time_begin(c, "build_top");
    k_build_top<<<(unsigned)c.top_bodies.size(), kThreads, 0, c.stream>>>(a);
    time_end(c, "build_top");
    ZQ_CUDA_TRY(cudaGetLastError());
  }
  return ZQ_OK;
}

}  // namespace zq
