// zq_tree.cu -- the bisection tree of Sec. 2.1 for m bodies at once.
//
// 1. per-body bounding box (the root box, normalised to side 1 per axis);
// 2. 21-bit quantisation and the bisection key: bit 62 - l of the key is the
//    half taken at bisection depth l (z, then y, then x per octree level);
// 3. per-body sort by (key, local bead index)  [zq_sort.cu];
// 4. LCP of neighbouring keys = depth of the bisection that separates them;
// 5. bottom-up construction: a node's parent is the neighbouring split with
//    the deeper (larger) LCP; each child deposits its far range end and its
//    height in the parent's 64-bit slot with one atomic exchange, and the
//    second to arrive completes the parent (range, count, height, residue
//    size 0/3/6 of Sec. 3) -- pruning of empty boxes and collapse of
//    single-child chains are implicit;
// 6. residue offsets by prefix sum over node ids (split-position order,
//    bodies concatenated);
// 7. the processing schedule: a stable bucket sort of the nodes by
//    (height, type) for heights up to the cut, the rest ("tail") last in
//    node-id order; node data is then re-laid out by slot.
#include "zq_internal.cuh"

namespace zq {

namespace {

constexpr int kThreads = 256;

__global__ void k_bead_body(const int64_t* __restrict__ off, int64_t m, int64_t N,
                            int32_t* __restrict__ bead_body) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) bead_body[i] = body_of_bead(off, m, i);
}

// Bounding boxes of all bodies (order-preserving integer encodings of the
// doubles, atomic min / max per body and axis) and the check for NaN and
// infinity.  A block takes kAabbItems beads per thread, consecutive beads
// per step (coalesced).  Bodies are contiguous, so a tile whose first and
// last bead belong to one body is that body's: thread-local min / max,
// one block reduction, three atomics per bound.  Other tiles go bead by
// bead, a warp at a time (one atomic per warp when the warp is one body's).
constexpr int kAabbItems = 4;

__global__ void __launch_bounds__(kThreads) k_aabb(const double* __restrict__ x, const double* __restrict__ y,
                                                   const double* __restrict__ z,
                                                   const int32_t* __restrict__ bead_body, int64_t N,
                                                   unsigned long long* __restrict__ lo,
                                                   unsigned long long* __restrict__ hi,
                                                   int32_t* __restrict__ err) {
  __shared__ unsigned long long wmn[3][kThreads / 32], wmx[3][kThreads / 32];
  const int64_t t0 = (int64_t)blockIdx.x * kThreads * kAabbItems;
  if (t0 >= N) return;
  const int64_t t1 = t0 + kThreads * kAabbItems < N ? t0 + kThreads * kAabbItems : N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t jf = bead_body[t0], jl = bead_body[t1 - 1];
  bool bad = false;
  if (jf == jl) {
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
#pragma unroll
    for (int k = 0; k < kAabbItems; ++k) {
      const int64_t i = t0 + k * kThreads + threadIdx.x;
      if (i < t1) {
        const double p[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          bad |= ((unsigned long long)__double_as_longlong(p[a]) & 0x7ff0000000000000ull) ==
                 0x7ff0000000000000ull;
          const unsigned long long e = ord_encode(p[a]);
          mn[a] = e < mn[a] ? e : mn[a];
          mx[a] = e > mx[a] ? e : mx[a];
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {  // min and max separately: the neutral values differ
        const unsigned long long omn = __shfl_xor_sync(0xffffffffu, mn[a], d);
        const unsigned long long omx = __shfl_xor_sync(0xffffffffu, mx[a], d);
        mn[a] = omn < mn[a] ? omn : mn[a];
        mx[a] = omx > mx[a] ? omx : mx[a];
      }
      if (lane == 0) {
        wmn[a][warp] = mn[a];
        wmx[a][warp] = mx[a];
      }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      const int a = threadIdx.x;
      unsigned long long m0 = wmn[a][0], m1 = wmx[a][0];
      for (int w = 1; w < kThreads / 32; ++w) {
        m0 = wmn[a][w] < m0 ? wmn[a][w] : m0;
        m1 = wmx[a][w] > m1 ? wmx[a][w] : m1;
      }
      atomicMin(&lo[3 * jf + a], m0);
      atomicMax(&hi[3 * jf + a], m1);
    }
  } else {
    for (int k = 0; k < kAabbItems; ++k) {
      const int64_t i = t0 + k * kThreads + threadIdx.x;
      const bool mine = i < t1;
      const int32_t j = mine ? bead_body[i] : -1;
      const double p[3] = {mine ? x[i] : 0.0, mine ? y[i] : 0.0, mine ? z[i] : 0.0};
      const int32_t j0 = __shfl_sync(0xffffffffu, j, 0);
      const bool uniform = __all_sync(0xffffffffu, j == j0) && j0 >= 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (mine)
          bad |= ((unsigned long long)__double_as_longlong(p[a]) & 0x7ff0000000000000ull) ==
                 0x7ff0000000000000ull;
        const unsigned long long e = mine ? ord_encode(p[a]) : 0ull;
        if (uniform) {
          unsigned long long mn = e, mx = e;
#pragma unroll
          for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long omn = __shfl_xor_sync(0xffffffffu, mn, d);
            const unsigned long long omx = __shfl_xor_sync(0xffffffffu, mx, d);
            mn = omn < mn ? omn : mn;
            mx = omx > mx ? omx : mx;
          }
          if (lane == 0) {
            atomicMin(&lo[3 * j0 + a], mn);
            atomicMax(&hi[3 * j0 + a], mx);
          }
        } else if (mine) {
          atomicMin(&lo[3 * j + a], e);
          atomicMax(&hi[3 * j + a], e);
        }
      }
    }
  }
  if (bad) atomicOr(err, kErrNonFinite);
}

// Per body and axis: the quantiser's constants (axis_quant, zq_internal.cuh).
__global__ void k_body_scale(int64_t m, const unsigned long long* __restrict__ lo,
                             const unsigned long long* __restrict__ hi, AxisQuant* __restrict__ q) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * m) return;
  q[t] = axis_quant(ord_decode(lo[t]), ord_decode(hi[t]));
}

__global__ void k_count_table(double* __restrict__ tab) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= kCountTab) return;
  const double s = sqrt((double)n);
  tab[n] = s;
  tab[kCountTab + n] = n > 0 ? 1.0 / s : 0.0;
}

// Keys of the beads of bodies above kSmallSortMax (the per-body tree
// kernels compute their own).
__global__ void k_keys(const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, const int32_t* __restrict__ bead_body,
                       const int64_t* __restrict__ off, int64_t N,
                       const unsigned long long* __restrict__ lo,
                       const unsigned long long* __restrict__ hi, const AxisQuant* __restrict__ bq,
                       uint64_t* __restrict__ key) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int32_t j = bead_body[i];
  if (off[j + 1] - off[j] <= kSmallSortMax) return;
  uint32_t q[3];
  const double p[3] = {x[i], y[i], z[i]};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const AxisQuant aq = bq[3 * j + a];
    q[a] = aq.beta < 0 ? 0u : quantise_fma(p[a], aq, ord_decode(lo[3 * j + a]), ord_decode(hi[3 * j + a]));
  }
  key[i] = bead_key(q[0], q[1], q[2]);
}

// Depth of the bisection separating sorted neighbours s and s+1 of a body:
// 63 coordinate levels (key bit 62 - l) followed by 32 index levels.
__global__ void k_lcp(const int64_t* __restrict__ off, const int32_t* __restrict__ bead_body,
                      int64_t N, const uint64_t* __restrict__ skey, const int32_t* __restrict__ perm,
                      uint8_t* __restrict__ lcp) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // sorted position
  if (s >= N) return;
  const int32_t j = bead_body[s];
  if (s == off[j + 1] - 1) return;  // last bead of a body: no split after it
  if (off[j + 1] - off[j] <= kSmallSortMax) return;
  const int64_t o = off[j];
  const int64_t q = s - j;          // node of the split between s and s + 1
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

__global__ void k_bottom_up(const int64_t* __restrict__ off, const int32_t* __restrict__ bead_body,
                            int64_t N, const uint8_t* __restrict__ lcp, int32_t* __restrict__ cl,
                            int32_t* __restrict__ cr, int32_t* __restrict__ first,
                            int32_t* __restrict__ cnt, uint8_t* __restrict__ height,
                            unsigned long long* __restrict__ slot, int32_t* __restrict__ res,
                            int32_t* __restrict__ root) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int32_t j = bead_body[s];
  const int64_t o = off[j];
  const int32_t n = (int32_t)(off[j + 1] - o);
  if (n <= kSmallSortMax) return;
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
    const int32_t g = is_left ? r : l - 1;
    const int64_t q = nb + g;
    if (is_left) cl[q] = code;  // each child enters its own code (read after the kernel)
    else cr[q] = code;
    // the deposit: this child's far range end and height; the second child
    // to arrive completes q from it (the exchange carries the data, so no
    // fence or second read is needed)
    const unsigned long long mine = (1ull << 63) | ((unsigned long long)(uint32_t)(is_left ? l : r) << 8) |
                                    (unsigned)h;
    const unsigned long long other = atomicExch(&slot[q], mine);
    if (other == 0ull) break;  // the sibling completes q
    const int32_t end = (int32_t)((other >> 8) & 0x7fffffffull);
    const int32_t hs = (int32_t)(other & 0xff);
    const int32_t lo_ = is_left ? l : end;
    const int32_t hi_ = is_left ? end : r;
    // the sibling covers [g + 1, hi_] (right) or [lo_, g] (left): internal when longer than one bead
    const bool sib_internal = is_left ? (hi_ > g + 1) : (lo_ < g);
    h = 1 + (h > hs ? h : hs);
    height[q] = (uint8_t)h;
    cnt[q] = hi_ - lo_ + 1;
    first[q] = (int32_t)(o + lo_);
    res[q] = 3 * ((code >= 0) + (sib_internal ? 1 : 0));
    code = (int32_t)q;
    l = lo_;
    r = hi_;
  }
}

// ------------------------------------------------------- schedule
constexpr int kBItems = 16;
constexpr int kBTile = kThreads * kBItems;

__device__ inline int node_bucket(const uint8_t* __restrict__ height, const int32_t* __restrict__ cl,
                                  const int32_t* __restrict__ cr, int64_t q, int cut) {
  return bucket_of(height[q], (cl[q] >= 0) + (cr[q] >= 0), cut);
}

// Warp w of block k takes the nodes [k kBTile + w kBRounds 32, + kBRounds 32)
// in rounds of 32 consecutive ids (coalesced loads); lanes with the same
// bucket are ranked by ballots in lane order, so ids keep their order
// inside each bucket (a stable counting sort).
constexpr int kBWarps = kThreads / 32;
constexpr int kBRounds = kBTile / kThreads;
static_assert(kMaxBuckets <= 64, "bucket ids are 6-bit digits");

__device__ __forceinline__ void warp_bucket_counts(const uint8_t* __restrict__ height,
                                                   const int32_t* __restrict__ cl,
                                                   const int32_t* __restrict__ cr, int64_t nodes, int cut,
                                                   int64_t base, int32_t* __restrict__ wc) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kBRounds; ++r) {
    const int64_t q = base + r * 32 + lane;
    const bool v = q < nodes;
    const int b = v ? node_bucket(height, cl, cr, q, cut) : 0;
    const unsigned peers = digit_peers<6>(b, v);
    if (v && (peers & lt) == 0) wc[b] += __popc(peers);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kThreads)
k_bucket_count(const uint8_t* __restrict__ height, const int32_t* __restrict__ cl,
               const int32_t* __restrict__ cr, int64_t nodes, int cut, int nb,
               int32_t* __restrict__ hist, int64_t nblk) {
  __shared__ int32_t wc[kBWarps][kMaxBuckets];
  for (int i = threadIdx.x; i < kBWarps * kMaxBuckets; i += blockDim.x) (&wc[0][0])[i] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  warp_bucket_counts(height, cl, cr, nodes, cut, (int64_t)blockIdx.x * kBTile + warp * kBRounds * 32, wc[warp]);
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    int32_t t = 0;
#pragma unroll
    for (int w = 0; w < kBWarps; ++w) t += wc[w][b];
    hist[(int64_t)b * nblk + blockIdx.x] = t;
  }
}

// Stable scatter: nodes keep increasing id order inside each bucket.
__global__ void __launch_bounds__(kThreads)
k_bucket_scatter(const uint8_t* __restrict__ height, const int32_t* __restrict__ cl,
                 const int32_t* __restrict__ cr, int64_t nodes, int cut, int nb,
                 const int32_t* __restrict__ hist, int64_t nblk, int32_t* __restrict__ sid,
                 int32_t* __restrict__ slot_of, int32_t* __restrict__ bstart) {
  __shared__ int32_t wc[kBWarps][kMaxBuckets];
  if (blockIdx.x == 0) {  // first slot of each bucket (the first block's start in it), then the end
    for (int b = threadIdx.x; b < nb; b += blockDim.x) bstart[b] = hist[(int64_t)b * nblk];
    if (threadIdx.x == 0) bstart[nb] = (int32_t)nodes;
  }
  for (int i = threadIdx.x; i < kBWarps * kMaxBuckets; i += blockDim.x) (&wc[0][0])[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kBTile + warp * kBRounds * 32;
  warp_bucket_counts(height, cl, cr, nodes, cut, base, wc[warp]);
  __syncthreads();
  // first slot of (bucket b, warp w): the block's start in b, then the
  // counts of the warps before w
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    int32_t run = hist[(int64_t)b * nblk + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kBWarps; ++w) {
      const int32_t t = wc[w][b];
      wc[w][b] = run;
      run += t;
    }
  }
  __syncthreads();
  for (int r = 0; r < kBRounds; ++r) {
    const int64_t q = base + r * 32 + lane;
    const bool v = q < nodes;
    const int b = v ? node_bucket(height, cl, cr, q, cut) : 0;
    const unsigned peers = digit_peers<6>(b, v);
    if (v) {
      const int32_t pos = wc[warp][b] + __popc(peers & lt);
      sid[pos] = (int32_t)q;
      slot_of[q] = pos;
    }
    __syncwarp();
    if (v && (peers & lt) == 0) wc[warp][b] += __popc(peers);
    __syncwarp();
  }
}


// Per-slot data, once the build's slots and the segment schedule are both
// made.  Each slot gets its children with their bead counts, and a leaf
// child as the index of its bead's coordinates (the build then reads a
// child's state, its count-table entries and a leaf's coordinates in one
// round of loads), its height, and its node's record offset (position
// order, from the segment schedule).
__global__ void k_slot_data(int64_t nodes, const int32_t* __restrict__ sid,
                            const int32_t* __restrict__ slot_of, const int32_t* __restrict__ cl,
                            const int32_t* __restrict__ cr, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ cnt, const uint8_t* __restrict__ height,
                            const int32_t* __restrict__ pos_of, const int32_t* __restrict__ prw,
                            int4* __restrict__ sc, uint8_t* __restrict__ sheight, int32_t* __restrict__ srw) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nodes) return;
  const int32_t q = sid[s];
  const int32_t a = cl[q], b = cr[q];
  srw[s] = prw[pos_of[q]];
  sc[s] = make_int4(a >= 0 ? slot_of[a] : -1 - perm[leaf_pos(a)], b >= 0 ? slot_of[b] : -1 - perm[leaf_pos(b)],
                    a >= 0 ? cnt[a] : 1, b >= 0 ? cnt[b] : 1);
  sheight[s] = height[q];
}


inline unsigned blocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

int64_t bucket_hist_words(int64_t nodes) {
  const int64_t nblk = (nodes + kBTile - 1) / kBTile;
  return kMaxBuckets * nblk + scan_tmp_words(kMaxBuckets * nblk);
}

zq_status launch_count_table(Ctx& c) {
  time_begin(c, "count_table");
  k_count_table<<<kCountTab / kThreads, kThreads, 0, c.stream>>>(c.count_tab);
  time_end(c, "count_table");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

zq_status launch_bead_body(Ctx& c) {
  time_begin(c, "bead_body");
  k_bead_body<<<blocks(c.N), kThreads, 0, c.stream>>>(c.off, c.m, c.N, c.bead_body);
  time_end(c, "bead_body");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

zq_status launch_tree(Ctx& c, const double* x, const double* y, const double* z, bool schedules) {
  cudaStream_t s = c.stream;
  unsigned long long* lo = reinterpret_cast<unsigned long long*>(c.aabb);
  unsigned long long* hi = lo + 3 * c.m;
  int32_t* err = c.counters + 2;
  // every body's bounding box in one pass over the coordinates (coalesced,
  // and it leaves them in L2 for the key pass)
  ZQ_CUDA_TRY(cudaMemsetAsync(lo, 0xff, 3 * c.m * sizeof(uint64_t), s));
  ZQ_CUDA_TRY(cudaMemsetAsync(hi, 0x00, 3 * c.m * sizeof(uint64_t), s));
  time_begin(c, "aabb");
  k_aabb<<<(unsigned)((c.N + kThreads * kAabbItems - 1) / (kThreads * kAabbItems)), kThreads, 0, s>>>(
      x, y, z, c.bead_body, c.N, lo, hi, err);
  time_end(c, "aabb");
  // bodies of at most kSmallSortMax beads: one thread block each
  zq_status st = launch_small_trees(c, x, y, z);
  if (st != ZQ_OK) return st;
  // larger bodies: device-wide kernels (they skip the beads of small bodies)
  if (!c.big_bodies.empty()) {
    time_begin(c, "keys");
    k_body_scale<<<blocks(3 * c.m), kThreads, 0, s>>>(c.m, lo, hi, c.body_q);
    time_end(c, "keys");
    time_begin(c, "keys");
    k_keys<<<blocks(c.N), kThreads, 0, s>>>(x, y, z, c.bead_body, c.off, c.N, lo, hi, c.body_q, c.key);
    time_end(c, "keys");
    ZQ_CUDA_TRY(cudaGetLastError());
    st = launch_sort(c);
    if (st != ZQ_OK) return st;
    time_begin(c, "lcp");
    k_lcp<<<blocks(c.N), kThreads, 0, s>>>(c.off, c.bead_body, c.N, c.skey, c.perm, c.lcp);
    time_end(c, "lcp");
    // one 64-bit deposit slot per node (the radix sort's ping-pong keys, free now)
    unsigned long long* slot = reinterpret_cast<unsigned long long*>(c.key_tmp);
    ZQ_CUDA_TRY(cudaMemsetAsync(slot, 0, c.nodes * sizeof(unsigned long long), s));
    time_begin(c, "bottom_up");
    k_bottom_up<<<blocks(c.N), kThreads, 0, s>>>(c.off, c.bead_body, c.N, c.lcp, c.cl, c.cr, c.first,
                                                 c.cnt, c.height, slot, c.roff, c.root);
    time_end(c, "bottom_up");
    ZQ_CUDA_TRY(cudaGetLastError());
  }
  if (!c.big_bodies.empty()) {  // else the per-body kernels wrote the offsets
    st = launch_exclusive_scan(c, c.roff, c.roff, c.nodes, c.scan_tmp, nullptr);
    if (st != ZQ_OK) return st;
  }
  c.have_sched = false;
  if (!schedules) return ZQ_OK;
  return launch_schedules(c);
}

zq_status launch_schedules(Ctx& c) {
  cudaStream_t s = c.stream;
  zq_status st = ZQ_OK;
  // The sweep schedule (segments) and the build schedule (buckets) only
  // read the tree: the former runs on a side stream next to the latter,
  // joined before the slot data, which needs both.
  ZQ_CUDA_TRY(cudaEventRecord(c.fork_ev, s));
  ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[1], c.fork_ev, 0));
  c.stream = c.side[1];
  st = launch_segments(c);
  c.stream = s;
  if (st != ZQ_OK) return st;
  ZQ_CUDA_TRY(cudaEventRecord(c.join_ev[1], c.side[1]));
  // schedule of the build
  const int nb = 3 * c.cut + 1;
  const int64_t nblk = (c.nodes + kBTile - 1) / kBTile;
  int32_t* hist = c.bhist;
  int32_t* tmp = c.bhist + kMaxBuckets * nblk;
  time_begin(c, "schedule");
  k_bucket_count<<<(unsigned)nblk, kThreads, 0, s>>>(c.height, c.cl, c.cr, c.nodes, c.cut, nb, hist, nblk);
  time_end(c, "schedule");
  st = launch_exclusive_scan(c, hist, hist, nb * nblk, tmp, nullptr);
  if (st != ZQ_OK) return st;
  time_begin(c, "schedule");
  k_bucket_scatter<<<(unsigned)nblk, kThreads, 0, s>>>(c.height, c.cl, c.cr, c.nodes, c.cut, nb, hist, nblk,
                                                      c.sid, c.slot_of, c.bstart);
  time_end(c, "schedule");
  ZQ_CUDA_TRY(cudaStreamWaitEvent(s, c.join_ev[1], 0));  // the segment schedule (positions, prw)
  time_begin(c, "schedule");
  k_slot_data<<<blocks(c.nodes), kThreads, 0, s>>>(c.nodes, c.sid, c.slot_of, c.cl, c.cr, c.perm, c.cnt,
                                                   c.height, c.pos_of, c.prw, c.sc, c.sheight, c.srw);
  time_end(c, "schedule");
  ZQ_CUDA_TRY(cudaGetLastError());
  c.have_sched = true;
  return ZQ_OK;
}

}  // namespace zq
