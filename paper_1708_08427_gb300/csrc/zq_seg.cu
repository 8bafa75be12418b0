// zq_seg.cu -- the segment schedule of the two sweeps.
//
// A segment is a maximal subtree with at most kSegMax beads (its root has
// at most kSegMax beads and is a body root or the child of a node with
// more).  Its internal nodes are the contiguous node-id range
// [first - j, first - j + count - 1) of body j (split positions of the
// subtree), so the segments and the nodes above them ("top" nodes) tile
// the node ids.  Positions: a top node keeps its id; the nodes of a segment
// are permuted inside the segment's id range so that heights increase
// (any order within one height).  The sweeps then take a segment per
// thread block, height by height, and the top nodes per body.
//
// Built after the tree, per call of zq_build_tree_batched; everything stays
// on the device (no host synchronisation): the number of segments is a
// device value that the grid-stride sweep kernels read.
#include "zq_internal.cuh"

namespace zq {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ bool seg_root_of(const int32_t* __restrict__ cnt, const int32_t* __restrict__ par,
                                            int64_t q) {
  if (cnt[q] > kSegMax) return false;
  const int32_t p = par[q];
  return p < 0 || cnt[p] > kSegMax;
}

// Parents; top nodes keep position = id.
__global__ void k_parents(int64_t nodes, const int32_t* __restrict__ cl, const int32_t* __restrict__ cr,
                          const int32_t* __restrict__ cnt, int32_t* __restrict__ par,
                          int32_t* __restrict__ pos_of, int32_t* __restrict__ pnode) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nodes) return;
  const int32_t a = cl[q], b = cr[q];
  if (a >= 0) par[a] = (int32_t)q;
  if (b >= 0) par[b] = (int32_t)q;
  if (cnt[q] > kSegMax) {
    pos_of[q] = (int32_t)q;
    pnode[q] = (int32_t)q;
  }
}

__global__ void k_seg_flags(int64_t nodes, const int32_t* __restrict__ cnt, const int32_t* __restrict__ par,
                            int32_t* __restrict__ flag) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nodes) flag[q] = seg_root_of(cnt, par, q) ? 1 : 0;
}

__global__ void k_seg_list(int64_t nodes, const int32_t* __restrict__ cnt, const int32_t* __restrict__ par,
                           const int32_t* __restrict__ idx, int4* __restrict__ seg) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nodes && seg_root_of(cnt, par, q)) seg[idx[q]] = make_int4((int32_t)q, 0, 0, 0);
}

__global__ void k_top_flags(int64_t nodes, const int32_t* __restrict__ cnt, int32_t* __restrict__ flag) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nodes) flag[q] = cnt[q] > kSegMax ? 1 : 0;
}

__global__ void k_top_list(int64_t nodes, const int32_t* __restrict__ cnt, const int32_t* __restrict__ idx,
                           int32_t* __restrict__ topv) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nodes && cnt[q] > kSegMax) topv[idx[q]] = (int32_t)q;
}

// top_off[j] = number of top nodes in bodies before j (node ids of body j
// start at off[j] - j); top_off[m] = all.
__global__ void k_top_off(int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ idx,
                          const int32_t* __restrict__ total, int32_t* __restrict__ top_off) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) top_off[j] = idx[off[j] - j];
  else if (j == m) top_off[m] = *total;
}

// One block per segment: body, range, and the height order inside it.
__global__ void __launch_bounds__(kThreads)
k_seg_order(const int32_t* __restrict__ nseg, int4* __restrict__ seg, const int64_t* __restrict__ off,
            int64_t m, const int32_t* __restrict__ first, const int32_t* __restrict__ cnt,
            const uint8_t* __restrict__ height, int32_t* __restrict__ pos_of, int32_t* __restrict__ pnode) {
  __shared__ int32_t hist[kMaxHeight + 1];
  __shared__ int4 info;
  const int ns = *nseg;
  for (int i = blockIdx.x; i < ns; i += gridDim.x) {
    if (threadIdx.x == 0) {
      const int32_t r = seg[i].x;
      const int32_t j = body_of_node(off, m, r);
      const int32_t f = first[r], c = cnt[r];
      info = make_int4(f - j, c - 1, f, c == (int32_t)(off[j + 1] - off[j]) ? 1 : 0);
      seg[i] = info;
    }
    for (int h = threadIdx.x; h <= kMaxHeight; h += blockDim.x) hist[h] = 0;
    __syncthreads();
    const int32_t a = info.x, nn = info.y;
    for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) atomicAdd(&hist[height[a + t]], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t run = 0;
      for (int h = 0; h <= kMaxHeight; ++h) {
        const int32_t v = hist[h];
        hist[h] = run;
        run += v;
      }
    }
    __syncthreads();
    for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) {
      const int32_t q = a + t;
      const int32_t p = a + atomicAdd(&hist[height[q]], 1);
      pos_of[q] = p;
      pnode[p] = q;
    }
    __syncthreads();
  }
}

// Per position: children as positions, residue offset, height and the
// record size in 4-word units (scanned into offsets afterwards).
__global__ void k_pos_data(int64_t nodes, const int32_t* __restrict__ pnode, const int32_t* __restrict__ pos_of,
                           const int32_t* __restrict__ cl, const int32_t* __restrict__ cr,
                           const int32_t* __restrict__ roff, const uint8_t* __restrict__ height,
                           int2* __restrict__ pc, int32_t* __restrict__ proff, uint8_t* __restrict__ ph,
                           int32_t* __restrict__ prw) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nodes) return;
  const int32_t q = pnode[p];
  const int32_t a = cl[q], b = cr[q];
  pc[p] = make_int2(a >= 0 ? pos_of[a] : a, b >= 0 ? pos_of[b] : b);
  proff[p] = roff[q];
  ph[p] = height[q];
  prw[p] = rec_words((a >= 0) + (b >= 0)) / 4;
}

}  // namespace

zq_status launch_segments(Ctx& c) {
  cudaStream_t s = c.stream;
  const int64_t n = c.nodes;
  ZQ_CUDA_TRY(cudaMemsetAsync(c.par, 0xff, n * sizeof(int32_t), s));
  time_begin(c, "segments");
  k_parents<<<blocks(n), kThreads, 0, s>>>(n, c.cl, c.cr, c.cnt, c.par, c.pos_of, c.pnode);
  k_seg_flags<<<blocks(n), kThreads, 0, s>>>(n, c.cnt, c.par, c.seg_flag);
  time_end(c, "segments");
  ZQ_TRY_STATUS(launch_exclusive_scan(c, c.seg_flag, c.seg_flag, n, c.scan_tmp, c.nseg));
  time_begin(c, "segments");
  k_seg_list<<<blocks(n), kThreads, 0, s>>>(n, c.cnt, c.par, c.seg_flag, c.seg);
  k_top_flags<<<blocks(n), kThreads, 0, s>>>(n, c.cnt, c.seg_flag);
  time_end(c, "segments");
  ZQ_TRY_STATUS(launch_exclusive_scan(c, c.seg_flag, c.seg_flag, n, c.scan_tmp, c.nseg + 1));
  time_begin(c, "segments");
  k_top_list<<<blocks(n), kThreads, 0, s>>>(n, c.cnt, c.seg_flag, c.topv);
  k_top_off<<<blocks(c.m + 1), kThreads, 0, s>>>(c.m, c.off, c.seg_flag, c.nseg + 1, c.top_off);
  k_seg_order<<<c.num_sms * 8, kThreads, 0, s>>>(c.nseg, c.seg, c.off, c.m, c.first, c.cnt, c.height,
                                                 c.pos_of, c.pnode);
  k_pos_data<<<blocks(n), kThreads, 0, s>>>(n, c.pnode, c.pos_of, c.cl, c.cr, c.roff, c.height, c.pc,
                                            c.proff, c.ph, c.prw);
  time_end(c, "segments");
  ZQ_TRY_STATUS(launch_exclusive_scan(c, c.prw, c.prw, n, c.scan_tmp, c.prw + n));
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

}  // namespace zq
