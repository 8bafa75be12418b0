// zq_build.cu -- the per-node transforms of Sec. 3 over a whole batch
// (node code in zq_build_node.cuh).
//
// Schedule: heights 1..cut level by level over all bodies (one launch per
// height, nodes sorted by type inside a height), then the remaining nodes
// one thread block (or warp) per body.  A node's children are finished
// before it.
#include "zq_build_node.cuh"
#include "zq_internal.cuh"
#include "zq_real.cuh"

namespace zq {

namespace {

constexpr int kThreads = 256;
// The level kernel (heights 2..cut) needs 96 registers: blocks of 128 let
// five fit an SM (20 warps) where blocks of 256 fit two (16 warps).
constexpr int kLevelThreads = 128;
constexpr int kLevelBlocksPerSM = 5;


// Height 1 holds exactly the nodes with two leaf children (Case I): a
// kernel of its own, which needs far fewer registers than the Householder
// cases and so runs at full occupancy.
template <class R>
__global__ void __launch_bounds__(kThreads) k_build_case1(BuildArgs a) {
  const int32_t s0 = a.bstart[0], s1 = a.bstart[1];
  for (int64_t s = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < s1;
       s += (int64_t)gridDim.x * blockDim.x)
    node_case1<R>(a, s, a.sc[s], 4 * (int64_t)(uint32_t)a.srw[s]);
}

// Heights 2..cut: only nodes with at least one internal child (k = 6, 9).
template <class R>
__global__ void __launch_bounds__(kLevelThreads, kLevelBlocksPerSM) k_build_level(BuildArgs a, int h) {
  const int b0 = 3 * (h - 1);
  const int32_t s1 = a.bstart[b0 + 1], s2 = a.bstart[b0 + 2], s3 = a.bstart[b0 + 3];
  for (int64_t s = s1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < s3;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rw = 4 * (int64_t)(uint32_t)a.srw[s];
    if (s < s2) build_slot<R>(a, s, 1, rw);
    else build_slot<R>(a, s, 2, rw);
  }
}

// Nodes above the cut: one block per body, height by height.
template <class R>
__global__ void __launch_bounds__(kThreads) k_build_tail(BuildArgs a) {
  const int32_t j = blockIdx.x;
  const int bt = 3 * a.cut;
  const int32_t t0 = a.bstart[bt], t1 = a.bstart[bt + 1];
  int32_t lo, hi;
  id_range(a.sid, t0, t1, a.off[j] - j, a.off[j + 1] - (j + 1), &lo, &hi);
  if (lo == hi) return;
  __shared__ HeightSort S;
  const uint8_t* sh = a.sheight;
  const bool sorted = sort_by_height(hi - lo, [&](int32_t t) { return make_int2(lo + t, sh[lo + t]); }, S);
  for (int h = S.lim[0]; h <= S.lim[1]; ++h) {
    if (sorted) {
      for (int32_t k = S.hs[h] + threadIdx.x; k < S.hs[h + 1]; k += blockDim.x) {
        const int32_t s = S.ids[k];
        const int4 cc = a.sc[s];
        build_slot<R>(a, s, (cc.x >= 0) + (cc.y >= 0), 4 * (int64_t)(uint32_t)a.srw[s]);
      }
    } else {
      for (int32_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
        if (sh[s] != h) continue;
        const int4 cc = a.sc[s];
        build_slot<R>(a, s, (cc.x >= 0) + (cc.y >= 0), 4 * (int64_t)(uint32_t)a.srw[s]);
      }
    }
    __syncthreads();
  }
}

// Nodes above the cut when every body has at most 8192 beads: one warp per
// body, height by height (__syncwarp orders the lanes' state writes and
// reads).  Every body's upper chain runs at once instead of one launch per
// height, and a body's nodes above the cut fit a warp's few passes.  The
// body's tail slots (contiguous, node-id order) are sorted by height in
// shared memory when there are at most kWarpTailMax of them; otherwise the
// warp scans them at every height.
constexpr int kTailWarps = 4;
constexpr int kWarpTailMax = 256;

template <class R>
__global__ void __launch_bounds__(32 * kTailWarps) k_build_tail_warp(BuildArgs a, int32_t m) {
  __shared__ int32_t ids[kTailWarps][kWarpTailMax];
  __shared__ int32_t hs[kTailWarps][kMaxHeight + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t j = blockIdx.x * kTailWarps + warp;
  if (j >= m) return;  // whole warp
  const int bt = 3 * a.cut;
  const int32_t t0 = a.bstart[bt], t1 = a.bstart[bt + 1];
  int32_t lo, hi;
  id_range(a.sid, t0, t1, a.off[j] - j, a.off[j + 1] - (j + 1), &lo, &hi);
  const int32_t n = hi - lo;
  if (n == 0) return;
  const uint8_t* sh = a.sheight;
  int hmin = kMaxHeight + 1, hmax = 0;
  for (int32_t t = lane; t < n; t += 32) {
    const int h = sh[lo + t];
    hmin = min(hmin, h);
    hmax = max(hmax, h);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    hmin = min(hmin, __shfl_xor_sync(0xffffffffu, hmin, d));
    hmax = max(hmax, __shfl_xor_sync(0xffffffffu, hmax, d));
  }
  const bool sorted = n <= kWarpTailMax;
  if (sorted) {  // counting sort of the slots by height
    int32_t* H = hs[warp];
    for (int h = lane; h < kMaxHeight + 2; h += 32) H[h] = 0;
    __syncwarp();
    for (int32_t t = lane; t < n; t += 32) atomicAdd(&H[sh[lo + t]], 1);
    __syncwarp();
    if (lane == 0) {
      int32_t run = 0;
      for (int h = hmin; h <= hmax + 1; ++h) {
        const int32_t v = H[h];
        H[h] = run;
        run += v;
      }
    }
    __syncwarp();
    for (int32_t t = lane; t < n; t += 32) ids[warp][atomicAdd(&H[sh[lo + t]], 1)] = lo + t;
    __syncwarp();
    // H[h] is now the end of height h; the start is the end of the previous
  }
  for (int h = hmin; h <= hmax; ++h) {
    if (sorted) {
      const int32_t k0 = h == hmin ? 0 : hs[warp][h - 1], k1 = hs[warp][h];
      for (int32_t k = k0 + lane; k < k1; k += 32) {
        const int32_t s = ids[warp][k];
        const int4 cc = a.sc[s];
        build_slot<R>(a, s, (cc.x >= 0) + (cc.y >= 0), 4 * (int64_t)(uint32_t)a.srw[s]);
      }
    } else {
      for (int32_t s = lo + lane; s < hi; s += 32) {
        if (sh[s] != h) continue;
        const int4 cc = a.sc[s];
        build_slot<R>(a, s, (cc.x >= 0) + (cc.y >= 0), 4 * (int64_t)(uint32_t)a.srw[s]);
      }
    }
    __syncwarp();
  }
}

__global__ void k_count_table_dd(const double* __restrict__ tab, float2* __restrict__ tab2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * kCountTab) return;
  const dd v = dd_from_double(tab[i]);
  tab2[i] = make_float2(v.hi, v.lo);
}

template <class R>
zq_status run_build(Ctx& c, const BuildArgs& a, const std::function<zq_status()>& after_levels) {
  const int grid = c.num_sms * kLevelBlocksPerSM;
  // timing brackets: "build" around the whole transform build, and
  // "build_level" around all level launches (few event records in a
  // captured step)
  time_open(c, "build");
  time_begin(c, "build_level");
  k_build_case1<R><<<c.num_sms * 8, kThreads, 0, c.stream>>>(a);
  for (int h = 2; h <= c.cut; ++h) {
    ++c.launches;
    k_build_level<R><<<grid, kLevelThreads, 0, c.stream>>>(a, h);
  }
  time_end(c, "build_level");
  if (after_levels) ZQ_TRY_STATUS(after_levels());
  time_begin(c, "build_tail");
  if (c.big_bodies.empty())
    k_build_tail_warp<R><<<(unsigned)((c.m + kTailWarps - 1) / kTailWarps), 32 * kTailWarps, 0, c.stream>>>(
        a, (int32_t)c.m);
  else
    k_build_tail<R><<<(unsigned)c.m, kThreads, 0, c.stream>>>(a);
  time_end(c, "build_tail");
  time_end(c, "build");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

}  // namespace

zq_status launch_count_table_dd(Ctx& c) {
  time_begin(c, "count_table");
  k_count_table_dd<<<2 * kCountTab / kThreads, kThreads, 0, c.stream>>>(c.count_tab, c.count_tab2);
  time_end(c, "count_table");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

zq_status launch_build(Ctx& c, const double* x, const double* y, const double* z, int which,
                       const std::function<zq_status()>& after_levels) {
  BuildArgs a;
  a.x = x; a.y = y; a.z = z;
  a.off = c.off; a.perm = nullptr; a.sc = c.sc; a.cnt = nullptr; a.sheight = c.sheight; a.sid = c.sid;
  a.bstart = c.bstart; a.srw = c.srw; a.cut = c.cut;
  a.ctab = c.count_tab;
  a.ctab2 = c.count_tab2;
  a.st = c.st64;
  a.rec64 = (which & 1) ? c.rec64 : nullptr;
  a.rec32 = (which & 2) ? c.rec32 : nullptr;
  a.err = c.counters + 2;
  c.st_is_dd = c.build_dd;
  return c.build_dd ? run_build<dd>(c, a, after_levels) : run_build<double>(c, a, after_levels);
}

}  // namespace zq
