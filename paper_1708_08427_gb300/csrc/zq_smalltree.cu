// zq_smalltree.cu -- the whole bisection tree of a body of at most 8192
// beads in one thread block (Sec. 2.1, same readings as zq_tree.cu):
//   1. bounding box: read from the device-wide pass over all bodies
//      (k_aabb, order-preserving integer encodings of the doubles);
//   2. 21-bit quantisation and bisection keys (z, then y, then x per octree
//      level, most significant first);
//   3. stable LSD radix sort of (key, body-local index) in shared memory,
//      8-bit digits, warp-level ranks from ballots: kHighPasses passes over
//      the high 8 kHighPasses key bits, then each run of equal high bits
//      (beads in one cell of the first 8 kHighPasses / 3 octree levels; a
//      few beads on a shell) sorted by insertion; bodies with a run of more
//      than 32 such beads take all eight passes instead.  Equal keys keep
//      index order;
//   4. LCP of sorted neighbours (63 coordinate levels, then 32 index levels);
//   5. bottom-up construction: a node's parent is the neighbouring split
//      with the larger LCP; each child deposits (code, range end, height) in
//      the parent's 64-bit shared-memory slot with one atomic exchange, and
//      the child that finds the sibling's deposit completes the parent.
// Output: the same global node arrays as the device-wide path (perm, child
// codes, first, count, height, residue size, root); when the batch has no
// larger bodies, the residue offsets themselves (6.).
#include "zq_internal.cuh"

namespace zq {

namespace {

// Radix passes over the high key bits before the run fix-up.  Two passes
// (the first 5 1/3 octree levels) leave runs of at most about ten beads on
// the shells of up to 8192 beads; each pass costs about a quarter of the
// kernel.
#ifndef ZQ_SORT_HIGH_PASSES
#define ZQ_SORT_HIGH_PASSES 2
#endif
constexpr int kHighPasses = ZQ_SORT_HIGH_PASSES;
// (an even count: the sorted order ends in the first buffer)
static_assert(kHighPasses == 2 || kHighPasses == 4, "an even number of passes over at most the high half");
constexpr int kHighShift = 64 - 8 * kHighPasses;

struct SmallTreeArgs {
  const double* x;
  const double* y;
  const double* z;
  const unsigned long long* lo;  // bounding boxes (ordered-integer encodings), 3 per body
  const unsigned long long* hi;
  const int64_t* off;
  const int32_t* bodies;  // body ids of this size class
  int32_t* perm;
  int32_t* cl;
  int32_t* cr;
  int32_t* first;
  int32_t* cnt;
  uint8_t* height;
  int32_t* res;
  int32_t* root;
  int32_t* err;
  int final_roff;  // 1: write residue offsets (no device-wide scan follows)
};

// A finished node in 63 bits: left and right child (14 bits each: bit 13
// set for a leaf, then its body-local position, else the body-local split
// position), first position (13 bits), bead count (14 bits), height (8 bits).
__device__ __forceinline__ uint32_t local_code(int32_t code, int64_t o, int64_t nb) {
  return code < 0 ? (1u << 13) | (uint32_t)(-1 - code - o) : (uint32_t)(code - nb);
}

__device__ __forceinline__ int32_t global_code(uint32_t lc, int64_t o, int64_t nb) {
  return (lc >> 13) ? (int32_t)(-1 - (o + (lc & 0x1fffu))) : (int32_t)(nb + lc);
}

__device__ __forceinline__ unsigned long long pack_node(uint32_t lc, uint32_t rc, int first, int cnt, int h) {
  return (unsigned long long)lc | ((unsigned long long)rc << 14) | ((unsigned long long)first << 28) |
         ((unsigned long long)cnt << 41) | ((unsigned long long)h << 55);
}

__device__ __forceinline__ uint32_t unpack(unsigned long long pk, int at, int bits) {
  return (uint32_t)((pk >> at) & ((1ull << bits) - 1));
}

// 3 per internal child (k - 3 of Eq. 3.5)
__device__ __forceinline__ int32_t residue_size(unsigned long long pk) {
  return 3 * ((unpack(pk, 13, 1) ^ 1u) + (unpack(pk, 27, 1) ^ 1u));
}

// Block-wide exclusive scan of one int per thread (THREADS a multiple of 32).
template <int THREADS>
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* sh, int32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += t;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int32_t w = (lane < THREADS / 32) ? sh[lane] : 0;
    int32_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += t;
    }
    sh[lane] = wi - w;
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  const int32_t r = inc - v + sh[warp];
  if (total) *total = sh[32];
  __syncthreads();
  return r;
}

template <int MAXN, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_small_tree(SmallTreeArgs a) {
  constexpr int NW = THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* keyA = reinterpret_cast<uint64_t*>(smem);
  uint64_t* keyB = keyA + MAXN;
  uint16_t* idxA = reinterpret_cast<uint16_t*>(keyB + MAXN);
  uint16_t* idxB = idxA + MAXN;
  int32_t* whist = reinterpret_cast<int32_t*>(idxB + MAXN);  // [NW][256]
  __shared__ int32_t sh[33];
  __shared__ double lim[6];  // lo[3], hi[3]
  __shared__ AxisQuant aq[3];

  const int32_t j = a.bodies[blockIdx.x];
  const int64_t o = a.off[j];
  const int n = (int)(a.off[j + 1] - o);
  const int tid = threadIdx.x;

  // ---- 1. bounding box: from the device-wide pass (k_aabb), which also
  // checked the coordinates for NaN and infinity
  if (tid < 3) {
    const double l = ord_decode(a.lo[3 * j + tid]), h = ord_decode(a.hi[3 * j + tid]);
    lim[tid] = l;
    lim[3 + tid] = h;
    aq[tid] = axis_quant(l, h);
  }
  __syncthreads();

  // ---- 2. keys: one FP64 fused multiply-add per axis (the FP64 pipe runs
  // at 1/64 of the FP32 rate here, and every block of a launch starts with
  // this loop); the few beads near a cell boundary take the exact formula
  {
    const AxisQuant Q[3] = {aq[0], aq[1], aq[2]};
#pragma unroll 4
    for (int i = tid; i < n; i += THREADS) {
      const double p[3] = {a.x[o + i], a.y[o + i], a.z[o + i]};
      uint32_t q[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) q[c] = Q[c].beta < 0 ? 0u : quantise_fma(p[c], Q[c], lim[c], lim[3 + c]);
      keyA[i] = bead_key(q[0], q[1], q[2]);
      idxA[i] = (uint16_t)i;
    }
  }
  __syncthreads();

  // ---- 3. stable LSD radix sort, 8-bit digits; warp w owns the chunk
  // [w * PER_WARP, (w + 1) * PER_WARP) of the current order
  const int lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int per_warp = (n + NW - 1) / NW;
  __shared__ int long_run;
  int pass_lo = 8 - kHighPasses;  // first the high key bits only (see the fix-up below)
  for (;;) {
  uint64_t* kin = keyA;
  uint64_t* kout = keyB;
  uint16_t* iin = idxA;
  uint16_t* iout = idxB;
  for (int pass = pass_lo; pass < 8; ++pass) {
    const int shift = 8 * pass;
    for (int d = lane; d < 256; d += 32) whist[warp * 256 + d] = 0;
    __syncwarp();
    const int c0 = min(n, warp * per_warp);
    const int c1 = min(n, c0 + per_warp);
    // counts per digit of this warp's chunk
    for (int base = c0; base < c1; base += 32) {
      const int i = base + lane;
      const bool v = i < c1;
      const int dg = v ? (int)((kin[i] >> shift) & 0xff) : 256 + lane;
      const unsigned peers = digit_peers(dg, v);
      if (v && (peers & lt) == 0) whist[warp * 256 + dg] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // exclusive scan over (digit, warp): thread t owns digit-major entries
    // [t * (256 * NW / THREADS), ...)
    constexpr int E = 256 * NW / THREADS;
    int32_t loc[E];
    int32_t s = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int f = tid * E + e;        // flattened (digit, warp) index
      const int dg = f / NW, w = f % NW;
      loc[e] = whist[w * 256 + dg];
      s += loc[e];
    }
    int32_t run = block_excl_scan<THREADS>(s, sh, nullptr);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int f = tid * E + e;
      const int dg = f / NW, w = f % NW;
      whist[w * 256 + dg] = run;  // first output position of (digit, warp)
      run += loc[e];
    }
    __syncthreads();
    // scatter in chunk order (stable)
    for (int base = c0; base < c1; base += 32) {
      const int i = base + lane;
      const bool v = i < c1;
      uint64_t k = 0;
      uint16_t ix = 0;
      int dg = 256 + lane;
      if (v) {
        k = kin[i];
        ix = iin[i];
        dg = (int)((k >> shift) & 0xff);
      }
      const unsigned peers = digit_peers(dg, v);
      if (v) {
        const int pos = whist[warp * 256 + dg] + __popc(peers & lt);
        kout[pos] = k;
        iout[pos] = ix;
      }
      __syncwarp();
      if (v && (peers & lt) == 0) whist[warp * 256 + dg] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    uint64_t* tk = kin; kin = kout; kout = tk;
    uint16_t* ti = iin; iin = iout; iout = ti;
  }
  // after an even number of passes the sorted data is back in keyA / idxA
  if (pass_lo == 0) break;
  // Fix-up of the high-bit order: beads whose keys share the high bits are
  // in index order; each such run is sorted by the low bits (stable, so
  // equal keys keep index order).  A run longer than 32 beads sends the
  // body through all 8 passes instead.
  if (tid == 0) long_run = 0;
  __syncthreads();
  for (int p = tid; p < n; p += THREADS) {
    const uint64_t hk = keyA[p] >> kHighShift;
    if (p > 0 && (keyA[p - 1] >> kHighShift) == hk) continue;   // not a run start
    int L = 1;
    while (p + L < n && L <= 32 && (keyA[p + L] >> kHighShift) == hk) ++L;
    if (L == 1) continue;
    if (L > 32) {
      long_run = 1;
      continue;
    }
    for (int u = p + 1; u < p + L; ++u) {  // insertion sort by the low half
      const uint64_t k = keyA[u];
      const uint16_t ix = idxA[u];
      int v = u - 1;
      while (v >= p && keyA[v] > k) {
        keyA[v + 1] = keyA[v];
        idxA[v + 1] = idxA[v];
        --v;
      }
      keyA[v + 1] = k;
      idxA[v + 1] = ix;
    }
  }
  __syncthreads();
  if (!long_run) break;
  // back to index order, then the full sort
  for (int p = tid; p < n; p += THREADS) keyB[idxA[p]] = keyA[p];
  __syncthreads();
  for (int i = tid; i < n; i += THREADS) {
    keyA[i] = keyB[i];
    idxA[i] = (uint16_t)i;
  }
  __syncthreads();
  pass_lo = 0;
  }

  // ---- 4. permutation and LCP of neighbours
  uint8_t* lcp = reinterpret_cast<uint8_t*>(keyB);   // keyB is free now
  for (int p = tid; p < n; p += THREADS) {
    a.perm[o + p] = (int32_t)(o + idxA[p]);
    if (p < n - 1) {
      const uint64_t k1 = keyA[p], k2 = keyA[p + 1];
      int d;
      if (k1 != k2) d = __clzll((long long)(k1 ^ k2)) - 1;
      else d = 63 + __clz((int)((uint32_t)idxA[p] ^ (uint32_t)idxA[p + 1]));
      lcp[p] = (uint8_t)d;
    }
  }
  __syncthreads();

  // ---- 5. bottom-up construction (node id of split g: o - j + g).
  // slot[g] = 0 until a child arrives; a deposit is
  //   bit 63 valid | bits 24..55 child code | bits 8..23 range end | bits 0..7 height
  // The child that completes g overwrites slot[g] with g's packed node
  // (pack_node; nothing else touches slot[g] after its second deposit), and
  // the nodes go out to global memory in node order after the walk, so the
  // stores are coalesced instead of six scattered ones per node.
  // A lane takes one step of its walk per iteration; a lane whose walk has
  // ended (it arrived first at a node, or completed the root) takes the
  // next unprocessed leaf, so warps stay full while a few walks are long.
  __shared__ int next_leaf;
  unsigned long long* slot = reinterpret_cast<unsigned long long*>(keyA);  // keyA is free now
  for (int p = tid; p < n; p += THREADS) slot[p] = 0ull;
  if (tid == 0) next_leaf = THREADS;
  __syncthreads();
  const int64_t nb = o - j;
  int l = tid, r = tid, h = 0;
  int32_t code = -1 - (int32_t)(o + tid);
  bool busy = tid < n, more = true;
  while (__any_sync(0xffffffffu, busy || more)) {
    if (!busy && more) {
      const int leaf = atomicAdd(&next_leaf, 1);
      if (leaf < n) {
        l = r = leaf;
        h = 0;
        code = -1 - (int32_t)(o + leaf);
        busy = true;
      } else {
        more = false;
      }
    }
    if (!busy) continue;
    if (l == 0 && r == n - 1) {
      a.root[j] = code;
      busy = false;
      continue;
    }
    bool is_left;
    if (l == 0) is_left = true;
    else if (r == n - 1) is_left = false;
    else is_left = lcp[r] > lcp[l - 1];
    const int g = is_left ? r : l - 1;
    const unsigned long long mine = (1ull << 63) | ((unsigned long long)(uint32_t)code << 24) |
                                    ((unsigned long long)(is_left ? l : r) << 8) | (unsigned)h;
    const unsigned long long other = atomicExch(&slot[g], mine);
    if (other == 0ull) {  // the sibling completes g
      busy = false;
      continue;
    }
    const int32_t sib = (int32_t)(uint32_t)(other >> 24);
    const int end = (int)((other >> 8) & 0xffff);
    const int hs = (int)(other & 0xff);
    const int lo_ = is_left ? l : end;
    const int hi_ = is_left ? end : r;
    const int64_t q = nb + g;
    const int32_t lc = is_left ? code : sib;
    const int32_t rc = is_left ? sib : code;
    h = 1 + (h > hs ? h : hs);
    slot[g] = pack_node(local_code(lc, o, nb), local_code(rc, o, nb), lo_, hi_ - lo_ + 1, h);
    code = (int32_t)q;
    l = lo_;
    r = hi_;
  }

  __syncthreads();
  for (int g = tid; g < n - 1; g += THREADS) {
    const unsigned long long pk = slot[g];
    const int32_t lc = global_code(unpack(pk, 0, 14), o, nb), rc = global_code(unpack(pk, 14, 14), o, nb);
    const int64_t q = nb + g;
    a.cl[q] = lc;
    a.cr[q] = rc;
    a.first[q] = (int32_t)(o + unpack(pk, 28, 13));
    a.cnt[q] = unpack(pk, 41, 14);
    a.height[q] = (uint8_t)unpack(pk, 55, 8);
    if (!a.final_roff) a.res[q] = 3 * ((lc >= 0) + (rc >= 0));
  }

  // ---- 6. residue offsets (when every body of the batch is built here):
  // body j's residues start at 3 off[j] - 6 j; inside the body, an exclusive
  // prefix of the residue sizes in node-id order
  if (a.final_roff) {
    const int nn = n - 1;
    const int per = (nn + THREADS - 1) / THREADS;
    const int g0 = min(nn, tid * per), g1 = min(nn, g0 + per);
    int32_t sum = 0;
    for (int g = g0; g < g1; ++g) sum += residue_size(slot[g]);
    int32_t run = block_excl_scan<THREADS>(sum, sh, nullptr) + (int32_t)(3 * o - 6 * (int64_t)j);
    for (int g = g0; g < g1; ++g) {
      a.res[nb + g] = run;
      run += residue_size(slot[g]);
    }
  }
}

template <int MAXN, int THREADS>
constexpr size_t small_tree_smem() {
  return (size_t)MAXN * (8 + 8 + 2 + 2) + (size_t)(THREADS / 32) * 256 * 4;
}

template <int MAXN, int THREADS>
zq_status launch_class(Ctx& c, const SmallTreeArgs& a, const int32_t* bodies, int count, cudaStream_t s) {
  if (count <= 0) return ZQ_OK;
  constexpr size_t smem = small_tree_smem<MAXN, THREADS>();
  ZQ_CUDA_TRY(cudaFuncSetAttribute(k_small_tree<MAXN, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  SmallTreeArgs b = a;
  b.bodies = bodies;
  ++c.launches;
  k_small_tree<MAXN, THREADS><<<(unsigned)count, THREADS, smem, s>>>(b);
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

}  // namespace

int small_tree_class(int64_t n) { return n <= 1024 ? 0 : (n <= 2048 ? 1 : (n <= 4096 ? 2 : 3)); }

// Bodies of at most kSmallSortMax beads: c.small_d lists them grouped by
// size class (c.small_class_start, host).
zq_status launch_small_trees(Ctx& c, const double* x, const double* y, const double* z) {
  SmallTreeArgs a;
  a.x = x; a.y = y; a.z = z;
  a.lo = reinterpret_cast<const unsigned long long*>(c.aabb);
  a.hi = a.lo + 3 * c.m;
  a.off = c.off; a.bodies = nullptr; a.perm = c.perm; a.cl = c.cl; a.cr = c.cr; a.first = c.first;
  a.cnt = c.cnt; a.height = c.height; a.res = c.roff; a.root = c.root; a.err = c.counters + 2;
  a.final_roff = c.big_bodies.empty() ? 1 : 0;
  const int* cs = c.small_class_start;
  // The size classes are independent (disjoint bodies): the three smaller
  // ones run on side streams forked from the context stream, so their
  // blocks fill the SMs that the largest class leaves free; all join back
  // before anything that reads the tree.  One timing span covers the four.
  time_begin(c, "small_tree");
  --c.launches;  // time_begin counted a launch; launch_class counts each one
  ZQ_CUDA_TRY(cudaEventRecord(c.fork_ev, c.stream));
  for (int i = 0; i < 3; ++i) ZQ_CUDA_TRY(cudaStreamWaitEvent(c.side[i], c.fork_ev, 0));
  zq_status st;
  if ((st = launch_class<8192, 1024>(c, a, c.small_d + cs[3], cs[4] - cs[3], c.stream)) != ZQ_OK) return st;
  if ((st = launch_class<4096, 512>(c, a, c.small_d + cs[2], cs[3] - cs[2], c.side[0])) != ZQ_OK) return st;
  if ((st = launch_class<2048, 256>(c, a, c.small_d + cs[1], cs[2] - cs[1], c.side[1])) != ZQ_OK) return st;
  if ((st = launch_class<1024, 256>(c, a, c.small_d + cs[0], cs[1] - cs[0], c.side[2])) != ZQ_OK) return st;
  for (int i = 0; i < 3; ++i) {
    ZQ_CUDA_TRY(cudaEventRecord(c.join_ev[i], c.side[i]));
    ZQ_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev[i], 0));
  }
  time_end(c, "small_tree");
  return ZQ_OK;
}

}  // namespace zq
