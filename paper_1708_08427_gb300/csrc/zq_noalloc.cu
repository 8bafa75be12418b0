// zq_noalloc.cu -- zq_apply_Q_noalloc: Q~v for one small body without any
// device allocation.
//
// For callers that cannot allocate device memory at the point of the call
// (code that runs where cudaMalloc is unavailable or not allowed: inside a
// host framework that owns all device memory through its own allocator, a
// real-time loop with a fixed memory budget, or a plugin that receives only
// device pointers).  Everything the computation needs besides the caller's
// inputs and outputs lives in one file-scope device array of fixed size
// (kScratchBytes below), which every GPU that loads the library holds until
// the process exits.
//
// One thread block computes, for one body of 3 <= n <= ZQ_NOALLOC_MAX_BEADS
// beads: the bisection tree (same readings as the rest of the library:
// 21-bit keys, z/y/x bisection, ties by index), then, height by height, each
// node's FP64 transform (Case I closed form, or the Householder LQ of
// [T22_x | T22_y | K] with the LAPACK reflector convention, T22's diagonal
// made nonnegative and the numerical rank decision) immediately applied to
// the node's Info-set, writing the Residues to the output in the same order
// as zq_apply_Q.
#include <mutex>

#include "zq_internal.cuh"

namespace zq {
namespace {

constexpr int kNA = ZQ_NOALLOC_MAX_BEADS;  // beads
constexpr int kNAThreads = 256;
// The bitonic sort pads n to a power of two P <= kNA; bead indices are
// uint16 with 0xffff as padding, and the arrival slots carry a 16-bit range
// end; the static shared arrays (19 bytes per bead) must fit in 48 KB.
static_assert((kNA & (kNA - 1)) == 0, "ZQ_NOALLOC_MAX_BEADS must be a power of two");
static_assert(kNA < 65535, "bead indices and range ends are 16-bit");
static_assert(kNA <= 2048, "static shared memory of k_noalloc_apply_q is sized for at most 2048 beads");

// Scratch layout (per body of at most kNA beads; node arrays indexed by
// split position g in [0, n - 2]):
struct NAScratch {
  int32_t perm[kNA];
  int32_t cl[kNA], cr[kNA], first[kNA], cnt[kNA], height[kNA], roff[kNA];
  double st[kNA][9];    // centroid (3), T22 packed lower triangle (6)
  double info[kNA][6];  // Info-set [t; r]
};
constexpr size_t kScratchBytes = sizeof(NAScratch);

// The scratch every call shares.  Host code must not use this name as a
// device address: kernels receive the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__device__ __forceinline__ uint64_t na_spread3(uint32_t v) {
  uint64_t s = v & 0x1fffffull;
  s = (s | (s << 32)) & 0x1f00000000ffffull;
  s = (s | (s << 16)) & 0x1f0000ff0000ffull;
  s = (s | (s << 8)) & 0x100f00f00f00f00full;
  s = (s | (s << 4)) & 0x10c30c30c30c30c3ull;
  s = (s | (s << 2)) & 0x1249249249249249ull;
  return s;
}

__device__ __forceinline__ uint32_t na_quantise(double p, double lo, double hi) {
  if (!(hi > lo)) return 0u;
  const double t = __ddiv_rn(__dsub_rn(p, lo), __dsub_rn(hi, lo));
  const double s = floor(__dmul_rn(t, (double)(1u << kQBits)));
  const double top = (double)((1u << kQBits) - 1);
  return s >= top ? ((1u << kQBits) - 1) : (uint32_t)s;
}

// Householder LQ of the 3 x K matrix M = A^T (A given as K x 3), T22's
// diagonal made nonnegative: fills L (3 x 3 lower, packed) and the
// reflectors of G = D H3 H2 H1 (v[j] with v[j][j] = 1, tau[j], and the sign
// flips D as flip[j]); G itself is never formed.  K is a compile-time
// constant so that every array stays in registers.
template <int K>
__device__ __forceinline__ void na_lq(double (&A)[K][3], double* L, double (&v)[3][K], double (&tau)[3],
                                      bool (&flip)[3]) {
  int emax = -100000;
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (A[i][c] != 0.0 && ilogb(A[i][c]) > emax) emax = ilogb(A[i][c]);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    // numerical rank decision: a column whose entries (diagonal down) are
    // all more than 40 binary orders below M's largest is rounding noise
    bool noise = true;
#pragma unroll
    for (int i = j; i < K; ++i)
      if (A[i][j] != 0.0 && ilogb(A[i][j]) >= emax - 40) noise = false;
    if (noise) {
#pragma unroll
      for (int i = j; i < K; ++i) A[i][j] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) v[j][i] = 0.0;
    v[j][j] = 1.0;
    double xn2 = 0.0;
#pragma unroll
    for (int i = j + 1; i < K; ++i) xn2 += A[i][j] * A[i][j];
    tau[j] = 0.0;
    if (xn2 != 0.0) {
      const double al = A[j][j];
      const double norm = sqrt(al * al + xn2);
      const double be = (al >= 0.0) ? -norm : norm;
      tau[j] = (be - al) / be;
#pragma unroll
      for (int i = j + 1; i < K; ++i) v[j][i] = A[i][j] / (al - be);
      A[j][j] = be;
#pragma unroll
      for (int i = j + 1; i < K; ++i) A[i][j] = 0.0;
#pragma unroll
      for (int c = j + 1; c < 3; ++c) {
        double w = 0.0;
#pragma unroll
        for (int i = j; i < K; ++i) w += v[j][i] * A[i][c];
#pragma unroll
        for (int i = j; i < K; ++i) A[i][c] -= tau[j] * w * v[j][i];
      }
    }
  }
  // nonnegative diagonal of R: rows of R and of G flip together
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    flip[j] = A[j][j] < 0.0;
    if (flip[j]) {
#pragma unroll
      for (int c = j; c < 3; ++c) A[j][c] = -A[j][c];
    }
  }
  L[0] = A[0][0]; L[1] = A[0][1]; L[2] = A[1][1]; L[3] = A[0][2]; L[4] = A[1][2]; L[5] = A[2][2];
}

// One node of Eq. 3.5 with K = 6 (one internal child, block L1) or K = 9
// (blocks L1 = T22_x, L2 = T22_y): M = [L1 | L2 | K], K = sk [d]x, factorised
// into L, then u <- G u = D H3 H2 H1 u.
template <int K>
__device__ __forceinline__ void na_node(const double* L1, const double* L2, double sk, const double* d,
                                        double* L, double (&u)[K]) {
  double A[K][3];
  const double* Ls[2] = {L1, L2};
#pragma unroll
  for (int b = 0; b < K / 3 - 1; ++b) {
    const double* Lc = Ls[b];
    A[3 * b][0] = Lc[0]; A[3 * b][1] = Lc[1]; A[3 * b][2] = Lc[3];
    A[3 * b + 1][0] = 0.0; A[3 * b + 1][1] = Lc[2]; A[3 * b + 1][2] = Lc[4];
    A[3 * b + 2][0] = 0.0; A[3 * b + 2][1] = 0.0; A[3 * b + 2][2] = Lc[5];
  }
  constexpr int k0 = K - 3;
  A[k0][0] = sk * 0.0; A[k0][1] = sk * d[2]; A[k0][2] = sk * (-d[1]);
  A[k0 + 1][0] = sk * (-d[2]); A[k0 + 1][1] = sk * 0.0; A[k0 + 1][2] = sk * d[0];
  A[k0 + 2][0] = sk * d[1]; A[k0 + 2][1] = sk * (-d[0]); A[k0 + 2][2] = sk * 0.0;
  double v[3][K], tau[3];
  bool flip[3];
  na_lq<K>(A, L, v, tau, flip);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double w = 0.0;
#pragma unroll
    for (int i = j; i < K; ++i) w += v[j][i] * u[i];
    w *= tau[j];
#pragma unroll
    for (int i = j; i < K; ++i) u[i] -= w * v[j][i];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j)
    if (flip[j]) u[j] = -u[j];
}

__global__ void __launch_bounds__(kNAThreads)
k_noalloc_apply_q(NAScratch* __restrict__ S, int n, const double* __restrict__ x,
                  const double* __restrict__ y, const double* __restrict__ z,
                  const double* __restrict__ vin, double* __restrict__ out) {
  __shared__ uint64_t key[kNA];
  __shared__ uint16_t idx[kNA];
  __shared__ uint8_t lcp[kNA];
  __shared__ unsigned long long slot[kNA];
  __shared__ double red[kNAThreads / 32][6];
  __shared__ double lim[6];
  __shared__ int32_t part[kNAThreads / 32 + 1];
  __shared__ int hroot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ---- bounding box
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = tid; i < n; i += kNAThreads) {
    const double p[3] = {x[i], y[i], z[i]};
    for (int c = 0; c < 3; ++c) {
      mn[c] = fmin(mn[c], p[c]);
      mx[c] = fmax(mx[c], p[c]);
    }
  }
  for (int c = 0; c < 3; ++c)
    for (int d = 16; d > 0; d >>= 1) {
      mn[c] = fmin(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], d));
      mx[c] = fmax(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], d));
    }
  if (lane == 0)
    for (int c = 0; c < 3; ++c) {
      red[warp][c] = mn[c];
      red[warp][3 + c] = mx[c];
    }
  __syncthreads();
  if (tid < 6) {
    double r = red[0][tid];
    for (int w = 1; w < kNAThreads / 32; ++w) r = tid < 3 ? fmin(r, red[w][tid]) : fmax(r, red[w][tid]);
    lim[tid] = r;
  }
  __syncthreads();

  // ---- keys and sort by (key, index): bitonic network in shared memory
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = tid; i < P; i += kNAThreads) {
    if (i < n) {
      uint32_t q[3] = {na_quantise(x[i], lim[0], lim[3]), na_quantise(y[i], lim[1], lim[4]),
                       na_quantise(z[i], lim[2], lim[5])};
      key[i] = na_spread3(q[0]) | (na_spread3(q[1]) << 1) | (na_spread3(q[2]) << 2);
      idx[i] = (uint16_t)i;
    } else {
      key[i] = ~0ull;
      idx[i] = 0xffffu;
    }
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = tid; t < (P >> 1); t += kNAThreads) {
        const int a = 2 * t - (t & (stride - 1)), b = a + stride;
        const bool asc = (a & size) == 0;
        const uint64_t ka = key[a], kb = key[b];
        const uint16_t ia = idx[a], ib = idx[b];
        if (((ka > kb) || (ka == kb && ia > ib)) == asc) {
          key[a] = kb; key[b] = ka;
          idx[a] = ib; idx[b] = ia;
        }
      }
      __syncthreads();
    }
  for (int p = tid; p < n; p += kNAThreads) {
    S->perm[p] = idx[p];
    slot[p] = 0ull;  // arrival slots must start empty in every call
    if (p < n - 1) {
      const uint64_t k1 = key[p], k2 = key[p + 1];
      lcp[p] = (uint8_t)(k1 != k2 ? __clzll((long long)(k1 ^ k2)) - 1
                                  : 63 + __clz((int)((uint32_t)idx[p] ^ (uint32_t)idx[p + 1])));
    }
  }
  __syncthreads();

  // ---- bottom-up construction (as zq_smalltree.cu)
  for (int leaf = tid; leaf < n; leaf += kNAThreads) {
    int l = leaf, r = leaf, h = 0;
    int32_t code = -1 - leaf;
    for (;;) {
      if (l == 0 && r == n - 1) {
        hroot = h;
        break;
      }
      const bool is_left = (l == 0) || (r != n - 1 && lcp[r] > lcp[l - 1]);
      const int g = is_left ? r : l - 1;
      const unsigned long long mine = (1ull << 63) | ((unsigned long long)(uint32_t)code << 24) |
                                      ((unsigned long long)(is_left ? l : r) << 8) | (unsigned)h;
      const unsigned long long other = atomicExch(&slot[g], mine);
      if (other == 0ull) break;
      const int32_t sib = (int32_t)(uint32_t)(other >> 24);
      const int end = (int)((other >> 8) & 0xffff), hs = (int)(other & 0xff);
      const int lo_ = is_left ? l : end, hi_ = is_left ? end : r;
      const int32_t lc = is_left ? code : sib, rc = is_left ? sib : code;
      h = 1 + (h > hs ? h : hs);
      S->cl[g] = lc;
      S->cr[g] = rc;
      S->first[g] = lo_;
      S->cnt[g] = hi_ - lo_ + 1;
      S->height[g] = h;
      S->roff[g] = 3 * ((lc >= 0) + (rc >= 0));
      code = g;
      l = lo_;
      r = hi_;
    }
  }
  __syncthreads();

  // ---- residue offsets: exclusive prefix over split positions
  {
    const int per = (n - 1 + kNAThreads - 1) / kNAThreads;
    const int g0 = tid * per, g1 = min(n - 1, g0 + per);
    int32_t s = 0;
    for (int g = g0; g < g1; ++g) s += S->roff[g];
    int32_t inc = s;
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += t;
    }
    if (lane == 31) part[warp] = inc;
    __syncthreads();
    if (tid == 0) {
      int32_t acc = 0;
      for (int w = 0; w < kNAThreads / 32; ++w) {
        const int32_t t = part[w];
        part[w] = acc;
        acc += t;
      }
    }
    __syncthreads();
    int32_t run = part[warp] + inc - s;
    for (int g = g0; g < g1; ++g) {
      const int32_t v = S->roff[g];
      S->roff[g] = run;
      run += v;
    }
  }
  __syncthreads();

  // ---- height by height: node transform (FP64) and upward step
  for (int hh = 1; hh <= hroot; ++hh) {
    for (int g = tid; g < n - 1; g += kNAThreads) {
      if (S->height[g] != hh) continue;
      const int32_t cx = S->cl[g], cy = S->cr[g];
      double cX[3], cY[3], LX[6], LY[6], tX[3], tY[3], rX[3], rY[3];
      int nx, ny;
      if (cx < 0) {
        const int b = S->perm[-1 - cx];
        cX[0] = x[b]; cX[1] = y[b]; cX[2] = z[b];
        tX[0] = vin[b]; tX[1] = vin[n + b]; tX[2] = vin[2 * n + b];
        nx = 1;
      } else {
        for (int i = 0; i < 3; ++i) cX[i] = S->st[cx][i];
        for (int i = 0; i < 6; ++i) LX[i] = S->st[cx][3 + i];
        for (int i = 0; i < 3; ++i) { tX[i] = S->info[cx][i]; rX[i] = S->info[cx][3 + i]; }
        nx = S->cnt[cx];
      }
      if (cy < 0) {
        const int b = S->perm[-1 - cy];
        cY[0] = x[b]; cY[1] = y[b]; cY[2] = z[b];
        tY[0] = vin[b]; tY[1] = vin[n + b]; tY[2] = vin[2 * n + b];
        ny = 1;
      } else {
        for (int i = 0; i < 3; ++i) cY[i] = S->st[cy][i];
        for (int i = 0; i < 6; ++i) LY[i] = S->st[cy][3 + i];
        for (int i = 0; i < 3; ++i) { tY[i] = S->info[cy][i]; rY[i] = S->info[cy][3 + i]; }
        ny = S->cnt[cy];
      }
      const double dn = (double)(nx + ny);
      const double al = sqrt((double)nx / dn), be = sqrt((double)ny / dn);
      const double sk = sqrt((double)nx * (double)ny / dn);
      double d[3], cp[3], L[6], t[3], s3[3];
      for (int i = 0; i < 3; ++i) {
        d[i] = cX[i] - cY[i];
        cp[i] = ((double)nx * cX[i] + (double)ny * cY[i]) / dn;
        // upward step (Eq. 4.2): t = alpha t_x + beta t_y, s = beta t_x - alpha t_y
        t[i] = al * tX[i] + be * tY[i];
        s3[i] = be * tX[i] - al * tY[i];
      }
      double r[3];  // the node's rotational Info-set: first three rows of G u
      const int32_t ro = S->roff[g];
      if (cx < 0 && cy < 0) {  // Case I, Eqs. 3.9-3.10: G u with the explicit 3 x 3 G
        const double dd2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        for (int i = 0; i < 6; ++i) L[i] = 0.0;
        if (dd2 == 0.0) {
          for (int i = 0; i < 3; ++i) r[i] = s3[i];
        } else {
          const double dnorm = sqrt(dd2);
          const double hd[3] = {d[0] / dnorm, d[1] / dnorm, d[2] / dnorm};
          double g1[3];
          if (d[1] != 0.0 || d[2] != 0.0) {
            const double sq = sqrt(d[1] * d[1] + d[2] * d[2]);
            g1[0] = 0.0; g1[1] = -d[2] / sq; g1[2] = d[1] / sq;
          } else {
            g1[0] = 0.0; g1[1] = 0.0; g1[2] = d[0] > 0.0 ? -1.0 : 1.0;
          }
          const double g2[3] = {hd[1] * g1[2] - hd[2] * g1[1], hd[2] * g1[0] - hd[0] * g1[2],
                                hd[0] * g1[1] - hd[1] * g1[0]};
          r[0] = g1[0] * s3[0] + g1[1] * s3[1] + g1[2] * s3[2];
          r[1] = g2[0] * s3[0] + g2[1] * s3[1] + g2[2] * s3[2];
          r[2] = -(hd[0] * s3[0] + hd[1] * s3[1] + hd[2] * s3[2]);
          const double sl = sk * dnorm;
          L[0] = sl * g2[0]; L[1] = sl * g2[1]; L[2] = -sl * g1[1];
          L[3] = sl * g2[2]; L[4] = -sl * g1[2]; L[5] = 0.0;
        }
      } else if (cx >= 0 && cy >= 0) {  // Eq. 3.5, k = 9: u = [r_x; r_y; s]
        double u[9] = {rX[0], rX[1], rX[2], rY[0], rY[1], rY[2], s3[0], s3[1], s3[2]};
        na_node<9>(LX, LY, sk, d, L, u);
        for (int i = 0; i < 3; ++i) r[i] = u[i];
        for (int i = 3; i < 9; ++i) out[ro + i - 3] = u[i];
      } else {                 // Case II, k = 6: u = [r_c; s] of the internal child c
        const double* Lc = cx >= 0 ? LX : LY;
        const double* rc = cx >= 0 ? rX : rY;
        double u[6] = {rc[0], rc[1], rc[2], s3[0], s3[1], s3[2]};
        na_node<6>(Lc, nullptr, sk, d, L, u);
        for (int i = 0; i < 3; ++i) r[i] = u[i];
        for (int i = 3; i < 6; ++i) out[ro + i - 3] = u[i];
      }
      for (int i = 0; i < 3; ++i) {
        S->st[g][i] = cp[i];
        S->info[g][i] = t[i];
        S->info[g][3 + i] = r[i];
      }
      for (int i = 0; i < 6; ++i) S->st[g][3 + i] = L[i];
    }
    __syncthreads();
  }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_noalloc_mu;
NAScratch* g_noalloc_ptr[64] = {nullptr};

}  // namespace
}  // namespace zq

extern "C" zq_status zq_apply_Q_noalloc(int device, void* cuda_stream, int64_t n, const double* x,
                                        const double* y, const double* z, const double* v, double* out) {
  using namespace zq;
  if (n < 3 || n > ZQ_NOALLOC_MAX_BEADS || !x || !y || !z || !v || !out || device < 0 || device >= 64)
    return ZQ_EINVAL;
  NAScratch* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
      int prev = 0;
      if (cudaGetDevice(&prev) != cudaSuccess) return ZQ_ECUDA;
      if (cudaSetDevice(device) != cudaSuccess) return ZQ_ECUDA;
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      cudaSetDevice(prev);
      if (e != cudaSuccess || !p) return ZQ_ECUDA;
      g_noalloc_ptr[device] = static_cast<NAScratch*>(p);
    }
    scratch = g_noalloc_ptr[device];
  }
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return ZQ_ECUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return ZQ_ECUDA;
  k_noalloc_apply_q<<<1, kNAThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      scratch, (int)n, x, y, z, v, out);
  const cudaError_t e = cudaGetLastError();
  if (prev != device) cudaSetDevice(prev);
  return e == cudaSuccess ? ZQ_OK : ZQ_ECUDA;
}
