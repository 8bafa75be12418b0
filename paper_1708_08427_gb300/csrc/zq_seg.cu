// zq_seg.cu -- the segment schedule of the two sweeps.
//
// A segment is a maximal subtree with at most kSegMax beads (its root has
// at most kSegMax beads and is a body root or the child of a node with
// more).  Its internal nodes are the contiguous node-id range
// [first - j, first - j + count - 1) of body j (split positions of the
// subtree), so the segments and the nodes above them ("top" nodes) tile
// the node ids.  Positions: a top node keeps its id; the nodes of a segment
// are permuted inside the segment's id range so that heights increase
// (any order within one height), which puts the segment root, the only
// node of the largest height, at the last position of the range.  The
// sweeps then take a segment per thread block, height by height, and the
// top nodes per body.
//
// Two kernels, both on the device (no host synchronisation:
// the number of segments is a device value that the grid-stride kernels
// read):
//   classify     per node: parents list their children that are segment
//                roots (and body roots list themselves) with the segment's
//                node range, first bead and residue offset; top nodes are
//                listed per body (body j's list lies in its own node-id
//                range [off[j] - j, ...), since a body has fewer top nodes
//                than internal nodes; the order inside a list is free, the
//                top-node sweeps order them by height) and get their
//                per-position data here (a child segment root sits at the
//                last position of its segment, which follows from its
//                count alone);
//   seg_order    one block per segment: height order, positions, and the
//                per-position data of its nodes.
// Record offsets need no scan: at a top node or the first position of a
// segment they have a closed form (rec_base), and inside a segment the
// block adds its nodes' record sizes in position order.
#include "zq_internal.cuh"

namespace zq {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// Appends the flagged lanes' segments (one atomic per warp; all 32 lanes
// of the warp must call): seg = (first node position, nodes, first sorted
// bead, whole body?), seg_r = residue offset of the first node.
__device__ __forceinline__ void warp_append(bool flag, int4 value, int32_t r, int32_t* __restrict__ count,
                                            int4* __restrict__ list, int32_t* __restrict__ list_r) {
  const unsigned b = __ballot_sync(0xffffffffu, flag);
  if (!b) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(b) - 1;
  int32_t base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(b));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (flag) {
    const int32_t i = base + __popc(b & ((1u << lane) - 1u));
    list[i] = value;
    list_r[i] = r;
  }
}

// The segment whose root is internal node c of body j (its nodes are the
// ids [first - j, first - j + count - 1)).
__device__ __forceinline__ int4 segment_of(int32_t c, int32_t j, bool whole, const int32_t* __restrict__ cnt,
                                           const int32_t* __restrict__ first, const int32_t* __restrict__ roff,
                                           int32_t* r) {
  const int32_t f = first[c], k = cnt[c];
  *r = roff[f - j];
  return make_int4(f - j, k - 1, f, whole ? 1 : 0);
}

// Record offset (4-word units) of position a when the positions before a
// are exactly the node ids before a (a top node keeps its id; a segment's
// positions permute its own id range).  A node's record takes 3 + (its
// internal children) units (rec_words).  A whole body j' of n beads
// contributes 3 (n - 1) + (n - 2) units (every node but the root is an
// internal child).  Inside body j, the splits g' < g (g = a - (off[j] - j))
// have g - delta internal children among their 2 g children: leaf i hangs
// from split i - 1 or split i, so the leaves 0..g-1, and leaf g when it is
// the right child of split g - 1 (delta = 1), are children of those splits.
// Together: 4 a - j - delta.
__device__ __forceinline__ int32_t rec_base(int64_t a, int32_t j, const int64_t* __restrict__ off,
                                            const int32_t* __restrict__ cr) {
  const int64_t g = a - (off[j] - j);
  const int delta = g > 0 && cr[a - 1] == (int32_t)(-1 - (off[j] + g));
  return (int32_t)(4 * a - j - delta);
}

// Position of a child code as the sweeps see it: a leaf stays a leaf, a
// top node keeps its id, a segment root is the last position of its range.
__device__ __forceinline__ int32_t child_pos(int32_t c, const int32_t* __restrict__ cnt,
                                             const int32_t* __restrict__ first,
                                             const int32_t* __restrict__ bead_body) {
  if (c < 0) return c;
  const int32_t k = cnt[c];
  if (k > kSegMax) return c;
  const int32_t f = first[c];
  return f - bead_body[f] + k - 2;
}

__global__ void k_classify(int64_t nodes, const int64_t* __restrict__ off, const int32_t* __restrict__ cl,
                           const int32_t* __restrict__ cr, const int32_t* __restrict__ cnt,
                           const int32_t* __restrict__ first, const int32_t* __restrict__ bead_body,
                           const int32_t* __restrict__ roff, const uint8_t* __restrict__ height,
                           int32_t* __restrict__ nseg, int4* __restrict__ seg, int32_t* __restrict__ seg_r,
                           int32_t* __restrict__ top_cnt, int32_t* __restrict__ topv,
                           int32_t* __restrict__ pos_of, int32_t* __restrict__ pnode, int2* __restrict__ pc,
                           int32_t* __restrict__ proff, uint8_t* __restrict__ ph, int32_t* __restrict__ prw,
                           int32_t rec_total) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) prw[nodes] = rec_total;
  bool self_root = false, left_root = false, right_root = false;
  int32_t a = -1, b = -1;
  int4 sq = make_int4(0, 0, 0, 0), sa = sq, sb = sq;
  int32_t rq = 0, ra = 0, rb = 0;
  if (q < nodes) {
    a = cl[q];
    b = cr[q];
    const int32_t c = cnt[q];
    const int32_t f = first[q];
    const int32_t j = bead_body[f];
    if (c <= kSegMax) {
      self_root = c == (int32_t)(off[j + 1] - off[j]);  // a whole body of at most kSegMax beads
      if (self_root) sq = segment_of((int32_t)q, j, true, cnt, first, roff, &rq);
    } else {
      left_root = a >= 0 && cnt[a] <= kSegMax;
      right_root = b >= 0 && cnt[b] <= kSegMax;
      if (left_root) sa = segment_of(a, j, false, cnt, first, roff, &ra);
      if (right_root) sb = segment_of(b, j, false, cnt, first, roff, &rb);
      topv[(int32_t)(off[j] - j) + atomicAdd(&top_cnt[j], 1)] = (int32_t)q;
      pos_of[q] = (int32_t)q;
      pnode[q] = (int32_t)q;
      pc[q] = make_int2(child_pos(a, cnt, first, bead_body), child_pos(b, cnt, first, bead_body));
      proff[q] = roff[q];
      ph[q] = height[q];
      prw[q] = rec_base(q, j, off, cr);
    }
  }
  warp_append(self_root, sq, rq, nseg, seg, seg_r);
  warp_append(left_root, sa, ra, nseg, seg, seg_r);
  warp_append(right_root, sb, rb, nseg, seg, seg_r);
}

// One block per segment: range, height order, positions, per-position data
// (blocks of 128: a segment averages a few hundred nodes).
constexpr int kOrderThreads = 128;

__global__ void __launch_bounds__(kOrderThreads)
k_seg_order(const int32_t* __restrict__ nseg, const int4* __restrict__ seg, const int64_t* __restrict__ off,
            const int32_t* __restrict__ bead_body, const int32_t* __restrict__ cl, const int32_t* __restrict__ cr,
            const int32_t* __restrict__ roff, const uint8_t* __restrict__ height, int32_t* __restrict__ pos_of,
            int32_t* __restrict__ pnode, int2* __restrict__ pc, int32_t* __restrict__ proff,
            uint8_t* __restrict__ ph, int32_t* __restrict__ prw) {
  constexpr int kPer = (kSegMax + kOrderThreads - 1) / kOrderThreads;
  __shared__ int32_t hist[kMaxHeight + 1];
  __shared__ int32_t units[kPer * kOrderThreads];  // record sizes by local position
  __shared__ int32_t wsum[kOrderThreads / 32];
  __shared__ int4 info;
  const int ns = *nseg;
  for (int i = blockIdx.x; i < ns; i += gridDim.x) {
    if (threadIdx.x == 0) info = seg[i];
    for (int h = threadIdx.x; h <= kMaxHeight; h += blockDim.x) hist[h] = 0;
    __syncthreads();
    const int32_t a = info.x, nn = info.y;
    for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) atomicAdd(&hist[height[a + t]], 1);
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the height counts by the first warp
      constexpr int kPer = (kMaxHeight + 1 + 31) / 32;
      const int lane = threadIdx.x, h0 = lane * kPer;
      int32_t v[kPer], t = 0;
#pragma unroll
      for (int e = 0; e < kPer; ++e) {
        v[e] = h0 + e <= kMaxHeight ? hist[h0 + e] : 0;
        t += v[e];
      }
      int32_t inc = t;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
      }
      int32_t run = inc - t;
#pragma unroll
      for (int e = 0; e < kPer; ++e) {
        if (h0 + e <= kMaxHeight) hist[h0 + e] = run;
        run += v[e];
      }
    }
    __syncthreads();
    for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) {
      const int32_t q = a + t;
      const int32_t p = a + atomicAdd(&hist[height[q]], 1);
      pos_of[q] = p;
      pnode[p] = q;
    }
    __syncthreads();  // pos_of of the whole segment is visible to the block
    for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) {
      const int32_t q = a + t;
      const int32_t l = cl[q], r = cr[q];
      const int32_t p = pos_of[q];
      pc[p] = make_int2(l >= 0 ? pos_of[l] : l, r >= 0 ? pos_of[r] : r);
      proff[p] = roff[q];
      ph[p] = height[q];
      units[p - a] = rec_words((l >= 0) + (r >= 0)) / 4;
    }
    __syncthreads();
    // record offsets: the closed form at the segment's first position, then
    // the sizes in position order (kPer consecutive positions per thread)
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      const int b0 = threadIdx.x * kPer;
      int32_t v[kPer], sum = 0;
#pragma unroll
      for (int e = 0; e < kPer; ++e) {
        v[e] = b0 + e < nn ? units[b0 + e] : 0;
        sum += v[e];
      }
      int32_t inc = sum;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
      }
      if (lane == 31) wsum[warp] = inc;
      __syncthreads();
      int32_t run = rec_base(a, bead_body[info.z], off, cr) + inc - sum;
      for (int w = 0; w < warp; ++w) run += wsum[w];
#pragma unroll
      for (int e = 0; e < kPer; ++e) {
        if (b0 + e < nn) prw[a + b0 + e] = run;
        run += v[e];
      }
    }
    __syncthreads();
  }
}

}  // namespace

zq_status launch_segments(Ctx& c) {
  cudaStream_t s = c.stream;
  const int64_t n = c.nodes, m = c.m;
  ZQ_CUDA_TRY(cudaMemsetAsync(c.nseg, 0, 2 * sizeof(int32_t), s));
  ZQ_CUDA_TRY(cudaMemsetAsync(c.top_cnt, 0, m * sizeof(int32_t), s));
  time_begin(c, "segments");
  k_classify<<<blocks(n), kThreads, 0, s>>>(n, c.off, c.cl, c.cr, c.cnt, c.first, c.bead_body, c.roff,
                                            c.height, c.nseg, c.seg, c.seg_r, c.top_cnt, c.topv, c.pos_of,
                                            c.pnode, c.pc, c.proff, c.ph, c.prw, (int32_t)(4 * n - m));
  k_seg_order<<<c.num_sms * 16, kOrderThreads, 0, s>>>(c.nseg, c.seg, c.off, c.bead_body, c.cl, c.cr, c.roff,
                                                       c.height, c.pos_of, c.pnode, c.pc, c.proff, c.ph, c.prw);
  time_end(c, "segments");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

}  // namespace zq
