// zq_tree.cu -- the bisection tree of Sec. 2.1 for m bodies at once.
//
// 1. per-body bounding box (the root box, normalised to side 1 per axis);
// 2. 21-bit quantisation and the bisection key: bit 62 - l of the key is the
//    half taken at bisection depth l (z, then y, then x per octree level);
// 3. per-body sort by (key, local bead index)  [zq_sort.cu];
// 4. LCP of neighbouring keys = depth of the bisection that separates them;
// 5. bottom-up construction: a node's parent is the neighbouring split with
//    the deeper (larger) LCP; the second child to arrive completes the
//    parent (range, count, height, residue size 0/3/6 of Sec. 3) -- pruning
//    of empty boxes and collapse of single-child chains are implicit;
// 6. residue offsets by prefix sum over node ids (split-position order,
//    bodies concatenated), and the tile / top classification of the sweeps.
#include "zq_internal.cuh"

namespace zq {

namespace {

constexpr int kThreads = 256;

__global__ void k_aabb(const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, const int64_t* __restrict__ off, int64_t m,
                       int64_t N, unsigned long long* __restrict__ lo,
                       unsigned long long* __restrict__ hi, int32_t* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool valid = i < N;
  const int32_t j = valid ? body_of_bead(off, m, i) : -1;
  double p[3] = {valid ? x[i] : 0.0, valid ? y[i] : 0.0, valid ? z[i] : 0.0};
  if (valid && !(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]))) atomicOr(err, kErrNonFinite);
  const int32_t j0 = __shfl_sync(0xffffffffu, j, 0);
  const bool uniform = __all_sync(0xffffffffu, j == j0) && j0 >= 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    unsigned long long e = valid ? ord_encode(p[a]) : 0ull;
    if (uniform) {
      unsigned long long mn = e, mx = e;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        unsigned long long omn = __shfl_xor_sync(0xffffffffu, mn, d);
        unsigned long long omx = __shfl_xor_sync(0xffffffffu, mx, d);
        mn = omn < mn ? omn : mn;
        mx = omx > mx ? omx : mx;
      }
      if (lane == 0) {
        atomicMin(&lo[3 * j0 + a], mn);
        atomicMax(&hi[3 * j0 + a], mx);
      }
    } else if (valid) {
      atomicMin(&lo[3 * j + a], e);
      atomicMax(&hi[3 * j + a], e);
    }
  }
}

// Spread the 21 low bits of v to every third bit (bit b -> bit 3b).
__device__ inline uint64_t spread3(uint32_t v) {
  uint64_t s = v & 0x1fffffull;
  s = (s | (s << 32)) & 0x1f00000000ffffull;
  s = (s | (s << 16)) & 0x1f0000ff0000ffull;
  s = (s | (s << 8)) & 0x100f00f00f00f00full;
  s = (s | (s << 4)) & 0x10c30c30c30c30c3ull;
  s = (s | (s << 2)) & 0x1249249249249249ull;
  return s;
}

// q = min(floor((p - lo) / (hi - lo) * 2^21), 2^21 - 1); 0 when hi == lo.
// Subtraction and division are IEEE correctly rounded; the product by 2^21
// is exact, so the result matches any IEEE implementation of the formula.
__device__ inline uint32_t quantise(double p, double lo, double hi) {
  if (!(hi > lo)) return 0u;
  double t = __ddiv_rn(__dsub_rn(p, lo), __dsub_rn(hi, lo));
  double s = floor(__dmul_rn(t, (double)(1u << kQBits)));
  const double top = (double)((1u << kQBits) - 1);
  return s >= top ? ((1u << kQBits) - 1) : (uint32_t)s;
}

__global__ void k_keys(const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, const int64_t* __restrict__ off, int64_t m,
                       int64_t N, const unsigned long long* __restrict__ lo,
                       const unsigned long long* __restrict__ hi, uint64_t* __restrict__ key) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int32_t j = body_of_bead(off, m, i);
  uint32_t q[3];
  const double p[3] = {x[i], y[i], z[i]};
#pragma unroll
  for (int a = 0; a < 3; ++a) q[a] = quantise(p[a], ord_decode(lo[3 * j + a]), ord_decode(hi[3 * j + a]));
  key[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
}

// Depth of the bisection separating sorted neighbours s and s+1 of a body:
// 63 coordinate levels (key bit 62 - l) followed by 32 index levels.
__global__ void k_lcp(const int64_t* __restrict__ off, int64_t m, int64_t nodes,
                      const uint64_t* __restrict__ skey, const int32_t* __restrict__ perm,
                      uint8_t* __restrict__ lcp) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nodes) return;
  const int32_t j = body_of_node(off, m, q);
  const int64_t o = off[j];
  const int64_t s = q + j;  // = o + (q - (o - j))
  const uint64_t k1 = skey[s], k2 = skey[s + 1];
  int d;
  if (k1 != k2) {
    d = __clzll((long long)(k1 ^ k2)) - 1;
  } else {
    uint32_t i1 = (uint32_t)(perm[s] - o), i2 = (uint32_t)(perm[s + 1] - o);
    d = 63 + __clz((int)(i1 ^ i2));
  }
  lcp[q] = (uint8_t)d;
}

__global__ void k_bottom_up(const int64_t* __restrict__ off, int64_t m, int64_t N,
                            const uint8_t* __restrict__ lcp, int32_t* __restrict__ cl,
                            int32_t* __restrict__ cr, int32_t* __restrict__ first,
                            int32_t* __restrict__ cnt, uint8_t* __restrict__ height,
                            int32_t* __restrict__ parent, int32_t* __restrict__ flag,
                            int32_t* __restrict__ res, int32_t* __restrict__ root) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int32_t j = body_of_bead(off, m, s);
  const int64_t o = off[j];
  const int32_t n = (int32_t)(off[j + 1] - o);
  const int64_t nb = o - j;
  int32_t l = (int32_t)(s - o), r = l;
  int32_t code = -1 - (int32_t)s;
  int32_t h = 0;
  for (;;) {
    if (l == 0 && r == n - 1) {
      root[j] = code;
      break;
    }
    bool is_left;
    if (l == 0) is_left = true;
    else if (r == n - 1) is_left = false;
    else is_left = lcp[nb + r] > lcp[nb + l - 1];
    const int64_t q = nb + (is_left ? r : l - 1);
    if (is_left) {
      cl[q] = code;
      first[q] = (int32_t)(o + l);
    } else {
      cr[q] = code;
      cnt[q] = r;  // the parent's last local position, until completion
    }
    if (code >= 0) parent[code] = (int32_t)q;
    __threadfence();
    if (atomicAdd(&flag[q], 1) == 0) break;  // the sibling completes q
    __threadfence();
    int32_t sib, lo_, hi_;
    if (is_left) {
      sib = __ldcg(&cr[q]);
      lo_ = l;
      hi_ = __ldcg(&cnt[q]);
    } else {
      sib = __ldcg(&cl[q]);
      lo_ = __ldcg(&first[q]) - (int32_t)o;
      hi_ = r;
    }
    const int32_t hs = is_leaf(sib) ? 0 : (int32_t)(*(volatile const uint8_t*)&height[sib]);
    h = 1 + (h > hs ? h : hs);
    height[q] = (uint8_t)h;
    cnt[q] = hi_ - lo_ + 1;
    res[q] = 3 * ((code >= 0) + (sib >= 0));
    code = (int32_t)q;
    l = lo_;
    r = hi_;
  }
}

__global__ void k_flags(const int32_t* __restrict__ cnt, const int32_t* __restrict__ parent,
                        int64_t nodes, int tile, int want_top, int32_t* __restrict__ f) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nodes) return;
  const int32_t c = cnt[q];
  int32_t v;
  if (want_top) {
    v = c > tile;
  } else {
    const int32_t p = parent[q];
    v = (c <= tile) && (p < 0 || cnt[p] > tile);
  }
  f[q] = v;
}

__global__ void k_compact(const int32_t* __restrict__ cnt, const int32_t* __restrict__ parent,
                          int64_t nodes, int tile, int want_top, const int32_t* __restrict__ pos,
                          int32_t* __restrict__ list) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nodes) return;
  const int32_t c = cnt[q];
  bool v;
  if (want_top) {
    v = c > tile;
  } else {
    const int32_t p = parent[q];
    v = (c <= tile) && (p < 0 || cnt[p] > tile);
  }
  if (v) list[pos[q]] = (int32_t)q;
}

inline unsigned blocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

zq_status launch_tree(Ctx& c, const double* x, const double* y, const double* z) {
  cudaStream_t s = c.stream;
  unsigned long long* lo = reinterpret_cast<unsigned long long*>(c.aabb);
  unsigned long long* hi = lo + 3 * c.m;
  int32_t* err = c.counters + 2;
  ZQ_CUDA_TRY(cudaMemsetAsync(lo, 0xff, 3 * c.m * sizeof(uint64_t), s));
  ZQ_CUDA_TRY(cudaMemsetAsync(hi, 0x00, 3 * c.m * sizeof(uint64_t), s));
  time_begin(c, "aabb");
  k_aabb<<<blocks(c.N), kThreads, 0, s>>>(x, y, z, c.off, c.m, c.N, lo, hi, err);
  time_end(c, "aabb");
  time_begin(c, "keys");
  k_keys<<<blocks(c.N), kThreads, 0, s>>>(x, y, z, c.off, c.m, c.N, lo, hi, c.key);
  time_end(c, "keys");
  ZQ_CUDA_TRY(cudaGetLastError());
  zq_status st = launch_sort(c);
  if (st != ZQ_OK) return st;
  time_begin(c, "lcp");
  k_lcp<<<blocks(c.nodes), kThreads, 0, s>>>(c.off, c.m, c.nodes, c.skey, c.perm, c.lcp);
  time_end(c, "lcp");
  ZQ_CUDA_TRY(cudaMemsetAsync(c.flag, 0, c.nodes * sizeof(int32_t), s));
  ZQ_CUDA_TRY(cudaMemsetAsync(c.parent, 0xff, c.nodes * sizeof(int32_t), s));
  time_begin(c, "bottom_up");
  k_bottom_up<<<blocks(c.N), kThreads, 0, s>>>(c.off, c.m, c.N, c.lcp, c.cl, c.cr, c.first, c.cnt,
                                               c.height, c.parent, c.flag, c.roff, c.root);
  time_end(c, "bottom_up");
  ZQ_CUDA_TRY(cudaGetLastError());
  st = launch_exclusive_scan(c, c.roff, c.roff, c.nodes, c.scan_tmp, nullptr);
  if (st != ZQ_OK) return st;
  for (int want_top = 0; want_top < 2; ++want_top) {
    time_begin(c, "classify");
    k_flags<<<blocks(c.nodes), kThreads, 0, s>>>(c.cnt, c.parent, c.nodes, c.tile, want_top, c.flag);
    time_end(c, "classify");
    st = launch_exclusive_scan(c, c.flag, c.flag, c.nodes, c.scan_tmp, c.counters + want_top);
    if (st != ZQ_OK) return st;
    time_begin(c, "classify");
    k_compact<<<blocks(c.nodes), kThreads, 0, s>>>(c.cnt, c.parent, c.nodes, c.tile, want_top, c.flag,
                                                   want_top ? c.top : c.tiles);
    time_end(c, "classify");
    ZQ_CUDA_TRY(cudaGetLastError());
  }
  return ZQ_OK;
}

}  // namespace zq
