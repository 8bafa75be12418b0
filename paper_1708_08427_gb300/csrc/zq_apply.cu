// zq_apply.cu -- the two sweeps.
//
// Upward (Q~ v, Algorithm 2, Eqs. 4.2-4.3): a leaf's Info-set is its bead
// vector f_i (Definition 4.1); every node turns its children's Info-sets
// into its own and writes its Residue (k - 3 numbers) at its residue
// offset.  Downward (Q~^T w, Algorithm 3, Theorem 4.3, Eqs. 4.6-4.7): the
// root Velocity-set is 0 (or given, for the whole Q); every node turns its
// Velocity-set and residue coefficients into its children's, and a leaf's
// velocity is the first three entries of its Velocity-set.  The node
// transforms are in zq_node.cuh.
//
// Schedule (zq_seg.cu): segments of at most kSegMax beads, one thread block
// per segment, height by height with the Info-/Velocity-sets in shared
// memory and the segment's bead values staged in shared memory; the nodes
// above the segments one thread block per body, through global memory.
// Upward: segments, then top nodes; downward: top nodes, then segments.
// The segment's records are prefetched into L2 in bulk when its block
// starts.
#include <cuda_bf16.h>

#include <type_traits>

#include "zq_internal.cuh"
#include "zq_node.cuh"

namespace zq {

namespace {

constexpr int kSegThreads = 128;
#ifndef ZQ_EARLY_SEG_BLOCKS
#define ZQ_EARLY_SEG_BLOCKS 6
#endif
constexpr int kEarlySegBlocksPerSM = ZQ_EARLY_SEG_BLOCKS;
constexpr int kTopThreads = 256;
// Bodies with at most this many top nodes: one warp each (k_*_top_warp);
// more: one thread block each (k_*_top).
constexpr int kWarpTop = 64;

template <typename T>
struct SweepArgs {
  int64_t N;
  const int32_t* perm;     // sorted position -> bead (null: vectors in tree order)
  const int2* pc;          // by position: children (positions or leaves)
  const int32_t* proff;    // residue offsets
  const uint8_t* ph;       // heights
  const uint32_t* prw;     // record offsets, 4-word units
  const int4* seg;         // segments
  const int32_t* seg_r;    // residue offset of each segment's first node
  const int32_t* nseg;     // device count of segments
  int64_t R;               // residues
  const int32_t* topv;     // top nodes of body j: [off[j] - j, off[j] - j + top_cnt[j])
  const int64_t* off;      // [m + 1] body bead offsets
  const int32_t* top_cnt;  // [m]
  const T* rec;
  T* xs;                   // Info-/Velocity-sets of segment roots and top nodes, by position
  const T* in;             // up: bead planes; down: residues
  T* out;                  // up: residues; down: bead planes
  const int32_t* bead_body;  // sorted position -> body
  T* root_out;             // up: the root Info-set [t; r] = Q_Z v per body (6 m), or null
  const T* root_in;        // down: the root Velocity-set per body (6 m), or null (zero)
  const double* rot;       // per body R_j (9 m, row-major), or null: bead vectors enter as
                           // R_j^T v_i (up) and leave as R_j L_i (down)
  int32_t cut;             // level cut of the build
  int seg_mode;            // upward: 0 all segments, 1 root height <= cut, 2 root height > cut
};

// A body's rotation in registers (on = false: the identity, nothing applied).
template <typename T>
struct Rot {
  T r[9];
  bool on;
};

// ROT = false (no rotations given) compiles the rotation away.
template <bool ROT, typename T>
__device__ __forceinline__ Rot<T> body_rot(const SweepArgs<T>& a, int64_t j) {
  Rot<T> R;
  R.on = ROT;
  if (ROT) {
#pragma unroll
    for (int k = 0; k < 9; ++k) R.r[k] = (T)__ldg(a.rot + 9 * j + k);
  }
  return R;
}

// v <- R^T v (a bead vector into the reference frame of the transforms)
template <typename T>
__device__ __forceinline__ void rot_in(const Rot<T>& R, T* v) {
  if (!R.on) return;
  const T a = v[0], b = v[1], c = v[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] = R.r[i] * a + R.r[3 + i] * b + R.r[6 + i] * c;
}

// v <- R v (a bead velocity out of the reference frame)
template <typename T>
__device__ __forceinline__ void rot_out(const Rot<T>& R, T* v) {
  if (!R.on) return;
  const T a = v[0], b = v[1], c = v[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] = R.r[3 * i] * a + R.r[3 * i + 1] * b + R.r[3 * i + 2] * c;
}

// ------------------------------------------------------------ helpers
// Bring [p, p + bytes) into L2 (bulk prefetch, 16-byte granules; chunks of
// at most 4 KB, one per thread of the first warp).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  const uint32_t chunks = (bytes + 4095u) / 4096u;
  for (uint32_t c = threadIdx.x; c < chunks; c += 32) {
    const uint32_t off = c * 4096u;
    const uint32_t len = min(4096u, bytes - off);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const char*>(p) + off),
                 "r"(len)
                 : "memory");
  }
}

// The same for the part of [p, p + bytes) that lies inside whole 16-byte
// granules of the array [base, base + limit) (the bulk prefetch takes
// 16-byte aligned ranges; nothing outside the array is touched).
__device__ __forceinline__ void prefetch_l2_inside(const void* base, int64_t limit, const void* p, int64_t bytes) {
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(base), b1 = b0 + (uintptr_t)limit;
  const uintptr_t p0 = reinterpret_cast<uintptr_t>(p);
  uintptr_t lo = p0 & ~(uintptr_t)15, hi = (p0 + (uintptr_t)bytes + 15) & ~(uintptr_t)15;
  const uintptr_t in_lo = (b0 + 15) & ~(uintptr_t)15, in_hi = b1 & ~(uintptr_t)15;
  lo = lo < in_lo ? in_lo : lo;
  hi = hi > in_hi ? in_hi : hi;
  if (hi > lo) prefetch_l2(reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo));
}

// One node's record (at most 80 bytes, 16-byte aligned) into L2: the
// lines holding its first word and the kRecMax-th (inside the record
// buffer, which holds kRecMax words per node).
template <typename T>
__device__ __forceinline__ void prefetch_l2_line(const T* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p + kRecMax - 1));
}

// Height boundaries of a segment: hb[h] = first local index of height h,
// hb[H + 1] = nn (the heights 1..H of a subtree are all present).  Returns H.
// Stages the segment's per-node data (children, record offset, residue
// offset, height) into shared memory in one coalesced pass, then the
// height boundaries.
struct SegMeta {
  int2 pc[kSegMax - 1];
  uint32_t rw[kSegMax - 1];
  int32_t ro[kSegMax - 1];
  uint8_t h[kSegMax - 1];
  int32_t hb[kMaxHeight + 2];
};

template <typename T>
__device__ __forceinline__ int stage_meta(const SweepArgs<T>& a, int32_t p0, int32_t nn, SegMeta& M) {
  for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) {
    M.pc[t] = a.pc[p0 + t];
    M.rw[t] = a.prw[p0 + t];
    M.ro[t] = a.proff[p0 + t];
    M.h[t] = a.ph[p0 + t];
  }
  __syncthreads();
  for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) {
    const int h = M.h[t];
    const int hp = t > 0 ? M.h[t - 1] : 0;
    for (int x = hp + 1; x <= h; ++x) M.hb[x] = t;
    if (t == nn - 1) M.hb[h + 1] = nn;
  }
  __syncthreads();
  return M.h[nn - 1];
}

template <typename T>
__device__ __forceinline__ int rec_type(int2 cc) { return (cc.x >= 0) + (cc.y >= 0); }

// ------------------------------------------------------------ upward
template <typename T>
__device__ __forceinline__ void up_dispatch(const SweepArgs<T>& a, uint32_t rw, int32_t ro, int2 cc, const T* X,
                                            const T* Y, T* P) {
  const T* r = a.rec + 4 * (int64_t)rw;
  T* res = a.out + ro;
  const int type = rec_type<T>(cc);
  if (type == 0) up_node<T, 0>(r, X, Y, false, P, res);
  else if (type == 1) up_node<T, 1>(r, X, Y, cc.x >= 0, P, res);
  else up_node<T, 2>(r, X, Y, true, P, res);
}

// The blocks of a grid share a bulk L2 prefetch of an array of `bytes`:
// block k takes the k-th slice.
__device__ __forceinline__ void prefetch_l2_share(const void* base, int64_t bytes) {
  const int64_t slice = ((bytes + gridDim.x - 1) / gridDim.x + 15) & ~(int64_t)15;
  const int64_t lo = (int64_t)blockIdx.x * slice;
  if (lo < bytes)
    prefetch_l2_inside(base, bytes, static_cast<const char*>(base) + lo, bytes - lo < slice ? bytes - lo : slice);
}

template <typename T, bool ROT>
__global__ void __launch_bounds__(kSegThreads) k_up_seg(SweepArgs<T> a) {
  __shared__ T info[(kSegMax - 1) * 6];
  __shared__ T bead[kSegMax * 3];
  __shared__ SegMeta M;
  const int ns = *a.nseg;
  // the bead vectors and the position -> bead map are gathered segment by
  // segment: bring them into L2 once, all blocks together (a few tens of MB;
  // tree-ordered vectors have no map)
  if (threadIdx.x < 32) {
    prefetch_l2_share(a.in, 3 * a.N * (int64_t)sizeof(T));
    if (a.perm) prefetch_l2_share(a.perm, a.N * (int64_t)sizeof(int32_t));
  }
  for (int i = blockIdx.x; i < ns; i += gridDim.x) {
    const int4 sg = a.seg[i];
    const int32_t p0 = sg.x, nn = sg.y, f = sg.z;
    if (a.seg_mode != 0 && ((int)a.ph[p0 + nn - 1] <= a.cut) != (a.seg_mode == 1)) continue;  // the whole block
    if (threadIdx.x < 32) {
      const uint32_t w0 = a.prw[p0], w1 = a.prw[p0 + nn];
      prefetch_l2(a.rec + 4 * (int64_t)w0, (w1 - w0) * 4u * (uint32_t)sizeof(T));
    }
    const Rot<T> R = body_rot<ROT>(a, ROT ? a.bead_body[f] : 0);
    for (int32_t t = threadIdx.x; t <= nn; t += blockDim.x) {
      const int32_t b = a.perm ? a.perm[f + t] : f + t;
      T v[3] = {a.in[b], a.in[a.N + b], a.in[2 * a.N + b]};
      rot_in(R, v);
      bead[3 * t] = v[0];
      bead[3 * t + 1] = v[1];
      bead[3 * t + 2] = v[2];
    }
    const int H = stage_meta(a, p0, nn, M);
    for (int h = 1; h <= H; ++h) {
      for (int32_t t = M.hb[h] + threadIdx.x; t < M.hb[h + 1]; t += blockDim.x) {
        const int2 cc = M.pc[t];
        const T* X = cc.x >= 0 ? info + 6 * (cc.x - p0) : bead + 3 * (leaf_pos(cc.x) - f);
        const T* Y = cc.y >= 0 ? info + 6 * (cc.y - p0) : bead + 3 * (leaf_pos(cc.y) - f);
        T P[6];
        up_dispatch(a, M.rw[t], M.ro[t], cc, X, Y, P);
#pragma unroll
        for (int k = 0; k < 6; ++k) info[6 * t + k] = P[k];
      }
      __syncthreads();
    }
    if (!sg.w && threadIdx.x < 6) a.xs[6 * (int64_t)(p0 + nn - 1) + threadIdx.x] = info[6 * (nn - 1) + threadIdx.x];
    if (sg.w && a.root_out && threadIdx.x < 6)  // a whole body: its root Info-set is Q_Z v
      a.root_out[6 * (int64_t)a.bead_body[f] + threadIdx.x] = info[6 * (nn - 1) + threadIdx.x];
    __syncthreads();
  }
}

// Height range of body j's top nodes into lim[0..1]; returns false if none.
__device__ __forceinline__ bool top_range(const int32_t* __restrict__ topv, const uint8_t* __restrict__ ph,
                                          int32_t t0, int32_t t1, int* lim) {
  if (t0 == t1) return false;
  if (threadIdx.x == 0) {
    lim[0] = kMaxHeight;
    lim[1] = 0;
  }
  __syncthreads();
  for (int32_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const int h = ph[topv[t]];
    atomicMin(&lim[0], h);
    atomicMax(&lim[1], h);
  }
  __syncthreads();
  return true;
}

template <typename T>
__device__ __forceinline__ void load_bead(const SweepArgs<T>& a, int32_t code, T* v, const Rot<T>& R) {
  const int32_t b = a.perm ? a.perm[leaf_pos(code)] : leaf_pos(code);
  v[0] = a.in[b];
  v[1] = a.in[a.N + b];
  v[2] = a.in[2 * a.N + b];
  rot_in(R, v);
}

template <bool ROT, typename T>
__device__ __forceinline__ void up_top_node(const SweepArgs<T>& a, int32_t p, bool root, int32_t j) {
  const int2 cc = a.pc[p];
  T X[6], Y[6], P[6];
  if (cc.x >= 0 && cc.y >= 0) {
    load6(a.xs + 6 * (int64_t)cc.x, X);
    load6(a.xs + 6 * (int64_t)cc.y, Y);
  } else {
    const Rot<T> R = body_rot<ROT>(a, j);
    if (cc.x >= 0) load6(a.xs + 6 * (int64_t)cc.x, X); else load_bead(a, cc.x, X, R);
    if (cc.y >= 0) load6(a.xs + 6 * (int64_t)cc.y, Y); else load_bead(a, cc.y, Y, R);
  }
  up_dispatch(a, a.prw[p], a.proff[p], cc, X, Y, P);
  store6(a.xs + 6 * (int64_t)p, P);
  if (root && a.root_out) store6(a.root_out + 6 * (int64_t)j, P);  // Q_Z v of body j
}

// Body blockIdx.x's top nodes, height by height (sorted by height in
// shared memory; bodies with more than kHeightSorted top nodes scan their
// list at every height).
template <typename T, bool ROT>
__global__ void __launch_bounds__(kTopThreads) k_up_top(SweepArgs<T> a) {
  __shared__ HeightSort S;
  const int32_t j = blockIdx.x;
  const int32_t t0 = (int32_t)(a.off[j] - j), n = a.top_cnt[j];
  if (n <= kWarpTop) return;  // none, or few: k_up_top_warp
  const int32_t* list = a.topv + t0;
  const uint8_t* ph = a.ph;
  // the body's top records into L2 first (they are scattered among the
  // segments' records), so the height-by-height chain reads them from L2
  for (int32_t t = threadIdx.x; t < n; t += blockDim.x) prefetch_l2_line(a.rec + 4 * (int64_t)a.prw[list[t]]);
  const bool sorted = sort_by_height(n, [&](int32_t t) { const int32_t p = list[t]; return make_int2(p, ph[p]); }, S);
  for (int h = S.lim[0]; h <= S.lim[1]; ++h) {
    if (sorted) {
      for (int32_t k = S.hs[h] + threadIdx.x; k < S.hs[h + 1]; k += blockDim.x)
        up_top_node<ROT>(a, S.ids[k], h == S.lim[1], j);
    } else {
      for (int32_t t = threadIdx.x; t < n; t += blockDim.x)
        if (ph[list[t]] == h) up_top_node<ROT>(a, list[t], h == S.lim[1], j);
    }
    __syncthreads();
  }
}

// Bodies with at most kWarpTop top nodes: one warp per body, lane l taking
// the body's top nodes l and l + 32, height by height with a warp barrier
// in between (a node's children are finished at lower heights; __syncwarp
// orders the warp's global writes before the reads of the next height).
// The records and the children's Info-sets are fetched into L2 first.
template <typename T>
struct TopPair {
  int32_t p[2];
  int h[2];
  int hmin, hmax;
};

template <typename T>
__device__ __forceinline__ bool warp_top_setup(const SweepArgs<T>& a, int32_t j, TopPair<T>& tp, bool down) {
  const int lane = threadIdx.x & 31;
  const int32_t t0 = (int32_t)(a.off[j] - j), n = a.top_cnt[j];
  if (n == 0 || n > kWarpTop) return false;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int32_t t = lane + 32 * e;
    tp.p[e] = t < n ? a.topv[t0 + t] : -1;
    tp.h[e] = tp.p[e] >= 0 ? (int)a.ph[tp.p[e]] : -1;
    if (tp.p[e] >= 0) {
      prefetch_l2_line(a.rec + 4 * (int64_t)a.prw[tp.p[e]]);
      if (down) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.in + a.proff[tp.p[e]]));
    }
  }
  const int lo = min(tp.h[0] >= 0 ? tp.h[0] : kMaxHeight + 1, tp.h[1] >= 0 ? tp.h[1] : kMaxHeight + 1);
  tp.hmin = __reduce_min_sync(0xffffffffu, lo);
  tp.hmax = __reduce_max_sync(0xffffffffu, max(tp.h[0], tp.h[1]));
  return true;
}

template <typename T, bool ROT>
__global__ void __launch_bounds__(kTopThreads) k_up_top_warp(SweepArgs<T> a, int32_t m) {
  const int32_t j = blockIdx.x * (kTopThreads / 32) + (threadIdx.x >> 5);
  if (j >= m) return;
  TopPair<T> tp;
  if (!warp_top_setup(a, j, tp, false)) return;
  for (int h = tp.hmin; h <= tp.hmax; ++h) {
#pragma unroll
    for (int e = 0; e < 2; ++e)
      if (tp.h[e] == h) up_top_node<ROT>(a, tp.p[e], h == tp.hmax, j);
    __syncwarp();
  }
}

// ---------------------------------------------------------- downward
template <typename T>
__device__ __forceinline__ void down_dispatch(const SweepArgs<T>& a, uint32_t rw, int32_t ro, int2 cc,
                                              const T* Lp, T* Lx, T* Ly) {
  const T* r = a.rec + 4 * (int64_t)rw;
  const T* w = a.in + ro;
  const int type = rec_type<T>(cc);
  if (type == 0) down_node<T, 0>(r, Lp, w, false, Lx, Ly);
  else if (type == 1) down_node<T, 1>(r, Lp, w, cc.x >= 0, Lx, Ly);
  else down_node<T, 2>(r, Lp, w, true, Lx, Ly);
}

template <typename T>
__device__ __forceinline__ void store_bead(const SweepArgs<T>& a, int32_t code, const T* L, const Rot<T>& R) {
  const int32_t b = a.perm ? a.perm[leaf_pos(code)] : leaf_pos(code);
  T u[3] = {L[0], L[1], L[2]};
  rot_out(R, u);
  a.out[b] = u[0];
  a.out[a.N + b] = u[1];
  a.out[2 * a.N + b] = u[2];
}

template <bool ROT, typename T>
__device__ __forceinline__ void down_top_node(const SweepArgs<T>& a, int32_t p, bool root, int32_t j) {
  const int2 cc = a.pc[p];
  T Lp[6], Lx[6], Ly[6];
  if (root) {
#pragma unroll
    for (int k = 0; k < 6; ++k) Lp[k] = a.root_in ? a.root_in[6 * (int64_t)j + k] : T(0);
  } else {
    load6(a.xs + 6 * (int64_t)p, Lp);
  }
  down_dispatch(a, a.prw[p], a.proff[p], cc, Lp, Lx, Ly);
  if (cc.x >= 0 && cc.y >= 0) {
    store6(a.xs + 6 * (int64_t)cc.x, Lx);
    store6(a.xs + 6 * (int64_t)cc.y, Ly);
  } else {
    const Rot<T> R = body_rot<ROT>(a, j);
    if (cc.x >= 0) store6(a.xs + 6 * (int64_t)cc.x, Lx); else store_bead(a, cc.x, Lx, R);
    if (cc.y >= 0) store6(a.xs + 6 * (int64_t)cc.y, Ly); else store_bead(a, cc.y, Ly, R);
  }
}

// Runs first: for every body with top nodes, the root Velocity-set is 0,
// then the top nodes from the root down (the root: the only top node of
// the largest height).
template <typename T, bool ROT>
__global__ void __launch_bounds__(kTopThreads) k_down_top(SweepArgs<T> a) {
  __shared__ HeightSort S;
  const int32_t j = blockIdx.x;
  const int32_t t0 = (int32_t)(a.off[j] - j), n = a.top_cnt[j];
  if (n <= kWarpTop) return;  // none, or few: k_down_top_warp
  const int32_t* list = a.topv + t0;
  const uint8_t* ph = a.ph;
  // the body's top records and residue coefficients into L2 first (they
  // are scattered), so the height-by-height chain reads them from L2
  for (int32_t t = threadIdx.x; t < n; t += blockDim.x) {
    const int32_t p = list[t];
    prefetch_l2_line(a.rec + 4 * (int64_t)a.prw[p]);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.in + a.proff[p]));  // 3 or 6 values
  }
  const bool sorted = sort_by_height(n, [&](int32_t t) { const int32_t p = list[t]; return make_int2(p, ph[p]); }, S);
  const int hmax = S.lim[1];
  for (int h = hmax; h >= S.lim[0]; --h) {
    if (sorted) {
      for (int32_t k = S.hs[h] + threadIdx.x; k < S.hs[h + 1]; k += blockDim.x)
        down_top_node<ROT>(a, S.ids[k], h == hmax, j);
    } else {
      for (int32_t t = threadIdx.x; t < n; t += blockDim.x)
        if (ph[list[t]] == h) down_top_node<ROT>(a, list[t], h == hmax, j);
    }
    __syncthreads();
  }
}

template <typename T, bool ROT>
__global__ void __launch_bounds__(kTopThreads) k_down_top_warp(SweepArgs<T> a, int32_t m) {
  const int32_t j = blockIdx.x * (kTopThreads / 32) + (threadIdx.x >> 5);
  if (j >= m) return;
  TopPair<T> tp;
  if (!warp_top_setup(a, j, tp, true)) return;
  for (int h = tp.hmax; h >= tp.hmin; --h) {
#pragma unroll
    for (int e = 0; e < 2; ++e)
      if (tp.h[e] == h) down_top_node<ROT>(a, tp.p[e], h == tp.hmax, j);
    __syncwarp();
  }
}

template <typename T, bool ROT>
__global__ void __launch_bounds__(kSegThreads) k_down_seg(SweepArgs<T> a) {
  __shared__ T info[(kSegMax - 1) * 6];
  __shared__ SegMeta M;
  const int ns = *a.nseg;
  for (int i = blockIdx.x; i < ns; i += gridDim.x) {
    const int4 sg = a.seg[i];
    const int32_t p0 = sg.x, nn = sg.y;
    if (threadIdx.x < 32) {
      const uint32_t w0 = a.prw[p0], w1 = a.prw[p0 + nn];
      prefetch_l2(a.rec + 4 * (int64_t)w0, (w1 - w0) * 4u * (uint32_t)sizeof(T));
      // the segment's residue coefficients: 3 (nn - 1) values from seg_r
      prefetch_l2_inside(a.in, a.R * (int64_t)sizeof(T), a.in + a.seg_r[i], 3 * (int64_t)(nn - 1) * sizeof(T));
    }
    if (threadIdx.x < 6)
      info[6 * (nn - 1) + threadIdx.x] =
          sg.w ? (a.root_in ? a.root_in[6 * (int64_t)a.bead_body[sg.z] + threadIdx.x] : T(0))
               : a.xs[6 * (int64_t)(p0 + nn - 1) + threadIdx.x];
    const Rot<T> R = body_rot<ROT>(a, ROT ? a.bead_body[sg.z] : 0);
    const int H = stage_meta(a, p0, nn, M);
    for (int h = H; h >= 1; --h) {
      for (int32_t t = M.hb[h] + threadIdx.x; t < M.hb[h + 1]; t += blockDim.x) {
        const int2 cc = M.pc[t];
        T Lp[6], Lx[6], Ly[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Lp[k] = info[6 * t + k];
        down_dispatch(a, M.rw[t], M.ro[t], cc, Lp, Lx, Ly);
        if (cc.x >= 0) {
#pragma unroll
          for (int k = 0; k < 6; ++k) info[6 * (cc.x - p0) + k] = Lx[k];
        } else {
          store_bead(a, cc.x, Lx, R);
        }
        if (cc.y >= 0) {
#pragma unroll
          for (int k = 0; k < 6; ++k) info[6 * (cc.y - p0) + k] = Ly[k];
        } else {
          store_bead(a, cc.y, Ly, R);
        }
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------ block form
// k right-hand sides at once, rows of k contiguous values: bead planes
// V[(a N + i) k + c], residues out[r k + c].  Storage TS (float, bfloat16,
// double), arithmetic TC (float for float/bfloat16 with the FP32 records,
// double with the FP64 records).  Thread (node, column) pairs cover each
// height; every column of a node reads the same record (L1 broadcast).
// Info-/Velocity-sets of all nodes live in the context's block scratch
// xk[(position * 6 + e) k + c] (reserved by zq_reserve_block).
template <typename TS, typename TC>
struct BlockArgs {
  int64_t N;
  int32_t k;
  const int32_t* perm;
  const int2* pc;
  const int32_t* proff;
  const uint8_t* ph;
  const uint32_t* prw;
  const int4* seg;
  const int32_t* nseg;
  const int32_t* topv;
  const int64_t* off;
  const int32_t* top_cnt;
  const TC* rec;
  TC* xk;
  const TS* in;
  TS* out;
};

__device__ __forceinline__ float to_c(float x) { return x; }
__device__ __forceinline__ double to_c(double x) { return x; }
__device__ __forceinline__ float to_c(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename TS> __device__ __forceinline__ TS from_c(float x);
template <> __device__ __forceinline__ float from_c<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <typename TS> __device__ __forceinline__ TS from_c(double x);
template <> __device__ __forceinline__ double from_c<double>(double x) { return x; }

template <typename TS, typename TC>
__device__ __forceinline__ void blk_child_up(const BlockArgs<TS, TC>& a, int32_t code, int32_t col, TC* X) {
  if (code >= 0) {
    const TC* p = a.xk + (int64_t)code * 6 * a.k + col;
#pragma unroll
    for (int e = 0; e < 6; ++e) X[e] = p[(int64_t)e * a.k];
  } else {
    const int64_t b = a.perm ? a.perm[leaf_pos(code)] : leaf_pos(code);
#pragma unroll
    for (int e = 0; e < 3; ++e) X[e] = to_c(a.in[((int64_t)e * a.N + b) * a.k + col]);
  }
}

template <typename TS, typename TC>
__device__ __forceinline__ void blk_up_one(const BlockArgs<TS, TC>& a, int64_t p, int2 cc, uint32_t rw, int32_t ro,
                                           int32_t col) {
  TC X[6], Y[6], P[6], res[6];
  blk_child_up(a, cc.x, col, X);
  blk_child_up(a, cc.y, col, Y);
  const TC* r = a.rec + 4 * (int64_t)rw;
  const int type = (cc.x >= 0) + (cc.y >= 0);
  if (type == 0) up_node<TC, 0>(r, X, Y, false, P, res);
  else if (type == 1) up_node<TC, 1>(r, X, Y, cc.x >= 0, P, res);
  else up_node<TC, 2>(r, X, Y, true, P, res);
  for (int e = 0; e < 3 * type; ++e) a.out[((int64_t)ro + e) * a.k + col] = from_c<TS>(res[e]);
  TC* q = a.xk + p * 6 * a.k + col;
#pragma unroll
  for (int e = 0; e < 6; ++e) q[(int64_t)e * a.k] = P[e];
}

template <typename TS, typename TC>
__device__ __forceinline__ void blk_down_one(const BlockArgs<TS, TC>& a, int64_t p, int2 cc, uint32_t rw, int32_t ro,
                                             int32_t col, bool zero) {
  TC Lp[6], Lx[6], Ly[6], w[6];
  const TC* q = a.xk + p * 6 * a.k + col;
#pragma unroll
  for (int e = 0; e < 6; ++e) Lp[e] = zero ? TC(0) : q[(int64_t)e * a.k];
  const int type = (cc.x >= 0) + (cc.y >= 0);
  for (int e = 0; e < 3 * type; ++e) w[e] = to_c(a.in[((int64_t)ro + e) * a.k + col]);
  const TC* r = a.rec + 4 * (int64_t)rw;
  if (type == 0) down_node<TC, 0>(r, Lp, w, false, Lx, Ly);
  else if (type == 1) down_node<TC, 1>(r, Lp, w, cc.x >= 0, Lx, Ly);
  else down_node<TC, 2>(r, Lp, w, true, Lx, Ly);
  const int32_t ch[2] = {cc.x, cc.y};
  const TC* L[2] = {Lx, Ly};
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    if (ch[s2] >= 0) {
      TC* d = a.xk + (int64_t)ch[s2] * 6 * a.k + col;
#pragma unroll
      for (int e = 0; e < 6; ++e) d[(int64_t)e * a.k] = L[s2][e];
    } else {
      const int64_t b = a.perm ? a.perm[leaf_pos(ch[s2])] : leaf_pos(ch[s2]);
#pragma unroll
      for (int e = 0; e < 3; ++e) a.out[((int64_t)e * a.N + b) * a.k + col] = from_c<TS>(L[s2][e]);
    }
  }
}

template <typename TS, typename TC>
__device__ __forceinline__ int stage_meta_blk(const BlockArgs<TS, TC>& a, int32_t p0, int32_t nn, SegMeta& M) {
  for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) {
    M.pc[t] = a.pc[p0 + t];
    M.rw[t] = a.prw[p0 + t];
    M.ro[t] = a.proff[p0 + t];
    M.h[t] = a.ph[p0 + t];
  }
  __syncthreads();
  for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) {
    const int h = M.h[t];
    const int hp = t > 0 ? M.h[t - 1] : 0;
    for (int x = hp + 1; x <= h; ++x) M.hb[x] = t;
    if (t == nn - 1) M.hb[h + 1] = nn;
  }
  __syncthreads();
  return M.h[nn - 1];
}

template <typename TS, typename TC>
__global__ void __launch_bounds__(256) k_up_seg_blk(BlockArgs<TS, TC> a) {
  __shared__ SegMeta M;
  const int ns = *a.nseg;
  const int32_t k = a.k;
  for (int i = blockIdx.x; i < ns; i += gridDim.x) {
    const int4 sg = a.seg[i];
    const int32_t p0 = sg.x, nn = sg.y;
    const int H = stage_meta_blk(a, p0, nn, M);
    for (int h = 1; h <= H; ++h) {
      const int32_t b0 = M.hb[h], nh = M.hb[h + 1] - b0;
      for (int32_t idx = threadIdx.x; idx < nh * k; idx += blockDim.x) {
        const int32_t t = b0 + idx / k, col = idx - (idx / k) * k;
        blk_up_one(a, p0 + t, M.pc[t], M.rw[t], M.ro[t], col);
      }
      __syncthreads();
    }
    __syncthreads();
  }
}

template <typename TS, typename TC>
__global__ void __launch_bounds__(256) k_down_seg_blk(BlockArgs<TS, TC> a) {
  __shared__ SegMeta M;
  const int ns = *a.nseg;
  const int32_t k = a.k;
  for (int i = blockIdx.x; i < ns; i += gridDim.x) {
    const int4 sg = a.seg[i];
    const int32_t p0 = sg.x, nn = sg.y;
    const int H = stage_meta_blk(a, p0, nn, M);
    for (int h = H; h >= 1; --h) {
      const int32_t b0 = M.hb[h], nh = M.hb[h + 1] - b0;
      for (int32_t idx = threadIdx.x; idx < nh * k; idx += blockDim.x) {
        const int32_t t = b0 + idx / k, col = idx - (idx / k) * k;
        blk_down_one(a, p0 + t, M.pc[t], M.rw[t], M.ro[t], col, h == H && sg.w);
      }
      __syncthreads();
    }
    __syncthreads();
  }
}

template <typename TS, typename TC>
__global__ void __launch_bounds__(kTopThreads) k_up_top_blk(BlockArgs<TS, TC> a) {
  __shared__ int lim[2];
  const int32_t j = blockIdx.x;
  const int32_t t0 = (int32_t)(a.off[j] - j), t1 = t0 + a.top_cnt[j];
  if (!top_range(a.topv, a.ph, t0, t1, lim)) return;
  const int32_t k = a.k, nt = t1 - t0;
  for (int h = lim[0]; h <= lim[1]; ++h) {
    for (int32_t idx = threadIdx.x; idx < nt * k; idx += blockDim.x) {
      const int32_t p = a.topv[t0 + idx / k], col = idx - (idx / k) * k;
      if (a.ph[p] != h) continue;
      blk_up_one(a, p, a.pc[p], a.prw[p], a.proff[p], col);
    }
    __syncthreads();
  }
}

template <typename TS, typename TC>
__global__ void __launch_bounds__(kTopThreads) k_down_top_blk(BlockArgs<TS, TC> a) {
  __shared__ int lim[2];
  const int32_t j = blockIdx.x;
  const int32_t t0 = (int32_t)(a.off[j] - j), t1 = t0 + a.top_cnt[j];
  if (!top_range(a.topv, a.ph, t0, t1, lim)) return;
  const int32_t k = a.k, nt = t1 - t0;
  for (int h = lim[1]; h >= lim[0]; --h) {
    for (int32_t idx = threadIdx.x; idx < nt * k; idx += blockDim.x) {
      const int32_t p = a.topv[t0 + idx / k], col = idx - (idx / k) * k;
      if (a.ph[p] != h) continue;
      blk_down_one(a, p, a.pc[p], a.prw[p], a.proff[p], col, h == lim[1]);
    }
    __syncthreads();
  }
}

template <typename TS, typename TC>
BlockArgs<TS, TC> make_block_args(const Ctx& c, int32_t k, const TC* rec, const TS* in, TS* out) {
  BlockArgs<TS, TC> a;
  a.N = c.N; a.k = k; a.perm = c.tree_order ? nullptr : c.perm; a.pc = c.pc; a.proff = c.proff; a.ph = c.ph;
  a.prw = reinterpret_cast<const uint32_t*>(c.prw);
  a.seg = c.seg; a.nseg = c.nseg; a.topv = c.topv; a.off = c.off; a.top_cnt = c.top_cnt;
  a.rec = rec; a.xk = static_cast<TC*>(c.xblk); a.in = in; a.out = out;
  return a;
}

// ---------------------------------------- block form on tensor cores
// The node transform meets a dense block of k columns: per node, the
// product G U (up: U = [r_x?; r_y?; s], k_p x k) or G^T Z (down: Z =
// [L_p(4:6); w_p]) is a small matrix product, run on the tensor cores with
// warp-level mma.sync (one warp per node): G, zero-padded to 16 x 16, is
// the A operand; U or Z, in tiles of 8 columns, the B operand; FP32
// accumulation.  MMA = Tf32: operands rounded to TF32 (10-bit significand,
// m16n8k8, two k-steps); MMA = Bf16: operands rounded to bfloat16 (8-bit
// significand, m16n8k16).  The elementwise parts of the node step (t_p =
// alpha t_x + beta t_y, s, and the Velocity-set combination) stay in FP32.
// Fragment layouts (PTX ISA, mma.sync): g = lane / 4, t = lane % 4;
// C/D (16 x 8): (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1).
struct Tf32 {};
struct Bf16 {};

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// A fragments of the 16 x 16 matrix As (row-major, FP32 in shared memory).
template <class MMA>
struct AFrag {
  uint32_t r[8];
};

template <class MMA>
__device__ __forceinline__ void load_a(const float (*As)[16], AFrag<MMA>& f) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  if constexpr (std::is_same_v<MMA, Tf32>) {
    // m16n8k8: a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4); k-step s adds 8 s
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      f.r[4 * ks + 0] = to_tf32(As[g][8 * ks + t]);
      f.r[4 * ks + 1] = to_tf32(As[g + 8][8 * ks + t]);
      f.r[4 * ks + 2] = to_tf32(As[g][8 * ks + t + 4]);
      f.r[4 * ks + 3] = to_tf32(As[g + 8][8 * ks + t + 4]);
    }
  } else {
    // m16n8k16: a0 (g, 2t..2t+1), a1 (g+8, 2t..), a2 (g, 2t+8..), a3 (g+8, 2t+8..)
    f.r[0] = pack_bf16(As[g][2 * t], As[g][2 * t + 1]);
    f.r[1] = pack_bf16(As[g + 8][2 * t], As[g + 8][2 * t + 1]);
    f.r[2] = pack_bf16(As[g][2 * t + 8], As[g][2 * t + 9]);
    f.r[3] = pack_bf16(As[g + 8][2 * t + 8], As[g + 8][2 * t + 9]);
  }
}

// D = A B for B the 16 x 8 tile Bs (row-major, FP32 in shared memory).
template <class MMA>
__device__ __forceinline__ void mma_tile(const AFrag<MMA>& A, const float (*Bs)[8], float (&d)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  d[0] = d[1] = d[2] = d[3] = 0.0f;
  if constexpr (std::is_same_v<MMA, Tf32>) {
    // b0 (t, g), b1 (t+4, g); k-step s adds 8 s to the row
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const uint32_t b0 = to_tf32(Bs[8 * ks + t][g]), b1 = to_tf32(Bs[8 * ks + t + 4][g]);
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
          : "r"(A.r[4 * ks]), "r"(A.r[4 * ks + 1]), "r"(A.r[4 * ks + 2]), "r"(A.r[4 * ks + 3]), "r"(b0),
            "r"(b1));
    }
  } else {
    // b0 (2t..2t+1, g), b1 (2t+8..2t+9, g)
    const uint32_t b0 = pack_bf16(Bs[2 * t][g], Bs[2 * t + 1][g]);
    const uint32_t b1 = pack_bf16(Bs[2 * t + 8][g], Bs[2 * t + 9][g]);
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(A.r[0]), "r"(A.r[1]), "r"(A.r[2]), "r"(A.r[3]), "r"(b0), "r"(b1));
  }
}

// Per-warp shared tiles: the node's G (or G^T), one 8-column tile of the B
// operand, one of the product.
struct TcTiles {
  float A[16][16];
  float B[16][8];
  float C[16][8];
};

// G (transpose: G^T) of node record r (FP32, compact layout) into T.A,
// zero-padded: lane j < k_p builds column j as G e_j.
__device__ __forceinline__ void tc_form_g(const float* __restrict__ rec, int type, bool transpose, TcTiles& T) {
  const int lane = threadIdx.x & 31;
  const int kp = 3 + 3 * type;
  if (lane < 16) {
    float u[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) u[i] = (i == lane) ? 1.0f : 0.0f;
    if (lane < kp) {
      if (type == 0) {  // G row-major in words 2..10
#pragma unroll
        for (int i = 0; i < 3; ++i) u[i] = __ldg(rec + 2 + 3 * i + lane);
      } else if (type == 1) {
        float r[16];
        load_rec<float, 16>(rec, r);
        g6(r, u, false);
      } else {
        float r[20];
        load_rec<float, 20>(rec, r);
        g9(r, u, false);
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float gv = (lane < kp && i < kp) ? u[i < 9 ? i : 0] : 0.0f;
      if (transpose) T.A[lane][i] = gv;  // G^T (lane, i) = G (i, lane)
      else T.A[i][lane] = gv;
    }
  }
  __syncwarp();
}

// Value i (0..2) of a child's Info-set part t (rows 0-2, or r: rows 3-5)
// in column col; a leaf child's t is its bead vector.
template <typename TS>
__device__ __forceinline__ float tc_child(const BlockArgs<TS, float>& a, int32_t code, int row, int32_t col) {
  if (code >= 0) return a.xk[((int64_t)code * 6 + row) * a.k + col];
  const int64_t b = a.perm ? a.perm[leaf_pos(code)] : leaf_pos(code);
  return to_c(a.in[((int64_t)row * a.N + b) * a.k + col]);
}

// Upward step of node p for all k columns, one warp (Algorithm 2 on a block):
// t_p = alpha t_x + beta t_y, [r_p; eps_p] = G [r_x?; r_y?; beta t_x - alpha t_y].
template <class MMA, typename TS>
__device__ void tc_up_node(const BlockArgs<TS, float>& a, int64_t p, int2 cc, uint32_t rw, int32_t ro, TcTiles& T) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int type = (cc.x >= 0) + (cc.y >= 0), kp = 3 + 3 * type;
  const float* rec = a.rec + 4 * (int64_t)rw;
  tc_form_g(rec, type, false, T);
  AFrag<MMA> A;
  load_a<MMA>(T.A, A);
  const float al = __ldg(rec), be = __ldg(rec + 1);
  const int32_t ic = cc.x >= 0 ? cc.x : cc.y;  // the internal child of a k = 6 node
  for (int32_t col0 = 0; col0 < a.k; col0 += 8) {
    for (int e = lane; e < 128; e += 32) {
      const int row = e >> 3, cl = e & 7;
      const int32_t col = col0 + cl;
      float val = 0.0f;
      if (row < kp && col < a.k) {
        const int sr = row - (kp - 3);  // row of s, or < 0
        if (sr >= 0) val = be * tc_child(a, cc.x, sr, col) - al * tc_child(a, cc.y, sr, col);
        else if (type == 2) val = tc_child(a, row < 3 ? cc.x : cc.y, 3 + row % 3, col);
        else val = tc_child(a, ic, 3 + row, col);
      }
      T.B[row][cl] = val;
    }
    __syncwarp();
    float d[4];
    mma_tile<MMA>(A, T.B, d);
    T.C[g][2 * t] = d[0];
    T.C[g][2 * t + 1] = d[1];
    T.C[g + 8][2 * t] = d[2];
    T.C[g + 8][2 * t + 1] = d[3];
    __syncwarp();
    for (int e = lane; e < (kp + 3) * 8; e += 32) {
      const int row = e >> 3, cl = e & 7;
      const int32_t col = col0 + cl;
      if (col >= a.k) continue;
      if (row < 3) {
        a.xk[((int64_t)p * 6 + 3 + row) * a.k + col] = T.C[row][cl];
      } else if (row < kp) {
        a.out[((int64_t)ro + row - 3) * a.k + col] = from_c<TS>(T.C[row][cl]);
      } else {
        const int i = row - kp;
        a.xk[((int64_t)p * 6 + i) * a.k + col] = al * tc_child(a, cc.x, i, col) + be * tc_child(a, cc.y, i, col);
      }
    }
    __syncwarp();
  }
}

// Downward step of node p for all k columns, one warp (Algorithm 3 on a
// block): [a_x?; a_y?; sigma] = G^T [L_p(4:6); w_p],
// L_x = [alpha L_p(1:3) + beta sigma; a_x], L_y = [beta L_p(1:3) - alpha sigma; a_y].
template <class MMA, typename TS>
__device__ void tc_down_node(const BlockArgs<TS, float>& a, int64_t p, int2 cc, uint32_t rw, int32_t ro, bool zero,
                             TcTiles& T) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int type = (cc.x >= 0) + (cc.y >= 0), kp = 3 + 3 * type;
  const float* rec = a.rec + 4 * (int64_t)rw;
  tc_form_g(rec, type, true, T);
  AFrag<MMA> A;
  load_a<MMA>(T.A, A);
  const float al = __ldg(rec), be = __ldg(rec + 1);
  const float* Lp = a.xk + (int64_t)p * 6 * a.k;
  for (int32_t col0 = 0; col0 < a.k; col0 += 8) {
    for (int e = lane; e < 128; e += 32) {
      const int row = e >> 3, cl = e & 7;
      const int32_t col = col0 + cl;
      float val = 0.0f;
      if (row < kp && col < a.k) {
        if (row < 3) val = zero ? 0.0f : Lp[(int64_t)(3 + row) * a.k + col];
        else val = to_c(a.in[((int64_t)ro + row - 3) * a.k + col]);
      }
      T.B[row][cl] = val;
    }
    __syncwarp();
    float d[4];
    mma_tile<MMA>(A, T.B, d);
    T.C[g][2 * t] = d[0];
    T.C[g][2 * t + 1] = d[1];
    T.C[g + 8][2 * t] = d[2];
    T.C[g + 8][2 * t + 1] = d[3];
    __syncwarp();
    for (int e = lane; e < 96; e += 32) {  // (child, row, column): 2 x 6 x 8
      const int side = e / 48, row = (e % 48) >> 3, cl = e & 7;
      const int32_t col = col0 + cl;
      const int32_t code = side ? cc.y : cc.x;
      if (col >= a.k || (code < 0 && row >= 3)) continue;
      float val;
      if (row < 3) {
        const float lp = zero ? 0.0f : Lp[(int64_t)row * a.k + col];
        const float sg = T.C[kp - 3 + row][cl];
        val = side ? be * lp - al * sg : al * lp + be * sg;
      } else {
        // a_x: rows 0-2 of C; a_y: rows 3-5 (k = 9) or 0-2 (k = 6)
        val = T.C[(side && type == 2 ? 3 : 0) + row - 3][cl];
      }
      if (code >= 0) {
        a.xk[((int64_t)code * 6 + row) * a.k + col] = val;
      } else {
        const int64_t b = a.perm ? a.perm[leaf_pos(code)] : leaf_pos(code);
        a.out[((int64_t)row * a.N + b) * a.k + col] = from_c<TS>(val);
      }
    }
    __syncwarp();
  }
}

constexpr int kTcWarps = 8;

template <class MMA, typename TS>
__global__ void __launch_bounds__(32 * kTcWarps) k_up_seg_tc(BlockArgs<TS, float> a) {
  __shared__ SegMeta M;
  __shared__ TcTiles T[kTcWarps];
  const int ns = *a.nseg, warp = threadIdx.x >> 5;
  for (int i = blockIdx.x; i < ns; i += gridDim.x) {
    const int4 sg = a.seg[i];
    const int32_t p0 = sg.x, nn = sg.y;
    const int H = stage_meta_blk(a, p0, nn, M);
    for (int h = 1; h <= H; ++h) {
      for (int32_t t = M.hb[h] + warp; t < M.hb[h + 1]; t += kTcWarps)
        tc_up_node<MMA>(a, p0 + t, M.pc[t], M.rw[t], M.ro[t], T[warp]);
      __syncthreads();
    }
    __syncthreads();
  }
}

template <class MMA, typename TS>
__global__ void __launch_bounds__(32 * kTcWarps) k_down_seg_tc(BlockArgs<TS, float> a) {
  __shared__ SegMeta M;
  __shared__ TcTiles T[kTcWarps];
  const int ns = *a.nseg, warp = threadIdx.x >> 5;
  for (int i = blockIdx.x; i < ns; i += gridDim.x) {
    const int4 sg = a.seg[i];
    const int32_t p0 = sg.x, nn = sg.y;
    const int H = stage_meta_blk(a, p0, nn, M);
    for (int h = H; h >= 1; --h) {
      for (int32_t t = M.hb[h] + warp; t < M.hb[h + 1]; t += kTcWarps)
        tc_down_node<MMA>(a, p0 + t, M.pc[t], M.rw[t], M.ro[t], h == H && sg.w, T[warp]);
      __syncthreads();
    }
    __syncthreads();
  }
}

template <class MMA, typename TS>
__global__ void __launch_bounds__(32 * kTcWarps) k_up_top_tc(BlockArgs<TS, float> a) {
  __shared__ int lim[2];
  __shared__ TcTiles T[kTcWarps];
  const int32_t j = blockIdx.x, warp = threadIdx.x >> 5;
  const int32_t t0 = (int32_t)(a.off[j] - j), t1 = t0 + a.top_cnt[j];
  if (!top_range(a.topv, a.ph, t0, t1, lim)) return;
  for (int h = lim[0]; h <= lim[1]; ++h) {
    for (int32_t t = t0 + warp; t < t1; t += kTcWarps) {
      const int32_t p = a.topv[t];
      if (a.ph[p] == h) tc_up_node<MMA>(a, p, a.pc[p], a.prw[p], a.proff[p], T[warp]);
    }
    __syncthreads();
  }
}

template <class MMA, typename TS>
__global__ void __launch_bounds__(32 * kTcWarps) k_down_top_tc(BlockArgs<TS, float> a) {
  __shared__ int lim[2];
  __shared__ TcTiles T[kTcWarps];
  const int32_t j = blockIdx.x, warp = threadIdx.x >> 5;
  const int32_t t0 = (int32_t)(a.off[j] - j), t1 = t0 + a.top_cnt[j];
  if (!top_range(a.topv, a.ph, t0, t1, lim)) return;
  for (int h = lim[1]; h >= lim[0]; --h) {
    for (int32_t t = t0 + warp; t < t1; t += kTcWarps) {
      const int32_t p = a.topv[t];
      if (a.ph[p] == h) tc_down_node<MMA>(a, p, a.pc[p], a.prw[p], a.proff[p], h == lim[1], T[warp]);
    }
    __syncthreads();
  }
}

template <class MMA, typename TS>
zq_status run_block_tc(Ctx& c, bool up, int32_t k, const void* in, void* out) {
  BlockArgs<TS, float> a =
      make_block_args<TS, float>(c, k, c.rec32, static_cast<const TS*>(in), static_cast<TS*>(out));
  if (up) {
    time_begin(c, "up_seg_blk");
    k_up_seg_tc<MMA, TS><<<c.num_sms * 8, 32 * kTcWarps, 0, c.stream>>>(a);
    time_end(c, "up_seg_blk");
    time_begin(c, "up_top_blk");
    k_up_top_tc<MMA, TS><<<(unsigned)c.m, 32 * kTcWarps, 0, c.stream>>>(a);
    time_end(c, "up_top_blk");
  } else {
    time_begin(c, "down_top_blk");
    k_down_top_tc<MMA, TS><<<(unsigned)c.m, 32 * kTcWarps, 0, c.stream>>>(a);
    time_end(c, "down_top_blk");
    time_begin(c, "down_seg_blk");
    k_down_seg_tc<MMA, TS><<<c.num_sms * 8, 32 * kTcWarps, 0, c.stream>>>(a);
    time_end(c, "down_seg_blk");
  }
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

template <typename TS, typename TC>
zq_status run_block(Ctx& c, bool up, int32_t k, const TC* rec, const void* in, void* out) {
  BlockArgs<TS, TC> a = make_block_args<TS, TC>(c, k, rec, static_cast<const TS*>(in), static_cast<TS*>(out));
  if (up) {
    time_begin(c, "up_seg_blk");
    k_up_seg_blk<TS, TC><<<c.num_sms * 8, 256, 0, c.stream>>>(a);
    time_end(c, "up_seg_blk");
    time_begin(c, "up_top_blk");
    k_up_top_blk<TS, TC><<<(unsigned)c.m, kTopThreads, 0, c.stream>>>(a);
    time_end(c, "up_top_blk");
  } else {
    time_begin(c, "down_top_blk");
    k_down_top_blk<TS, TC><<<(unsigned)c.m, kTopThreads, 0, c.stream>>>(a);
    time_end(c, "down_top_blk");
    time_begin(c, "down_seg_blk");
    k_down_seg_blk<TS, TC><<<c.num_sms * 8, 256, 0, c.stream>>>(a);
    time_end(c, "down_seg_blk");
  }
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

template <typename T>
SweepArgs<T> make_args(const Ctx& c, const T* rec, T* xs, const T* in, T* out) {
  SweepArgs<T> a;
  a.N = c.N; a.perm = c.tree_order ? nullptr : c.perm; a.pc = c.pc; a.proff = c.proff; a.ph = c.ph;
  a.prw = reinterpret_cast<const uint32_t*>(c.prw);
  a.seg = c.seg; a.seg_r = c.seg_r; a.R = c.R; a.nseg = c.nseg; a.topv = c.topv; a.off = c.off; a.top_cnt = c.top_cnt;
  a.rec = rec; a.xs = xs; a.in = in; a.out = out;
  a.bead_body = c.bead_body; a.root_out = nullptr; a.root_in = nullptr; a.rot = nullptr;
  a.cut = c.cut; a.seg_mode = 0;
  return a;
}

template <typename T>
zq_status run_up(Ctx& c, const T* rec, T* xs, const T* v, T* out, T* root_out, const double* rot, int seg_mode) {
  SweepArgs<T> a = make_args<T>(c, rec, xs, v, out);
  a.root_out = root_out;
  a.rot = rot;
  a.seg_mode = seg_mode;
  // the early part runs beside the build's nodes above the cut: fewer
  // persistent blocks, so that the build's blocks still find room
  const unsigned grid = (unsigned)c.num_sms * (seg_mode == 1 ? kEarlySegBlocksPerSM : 16);
  time_begin(c, seg_mode == 1 ? "up_seg_early" : "up_seg");
  if (rot) k_up_seg<T, true><<<grid, kSegThreads, 0, c.stream>>>(a);
  else k_up_seg<T, false><<<grid, kSegThreads, 0, c.stream>>>(a);
  time_end(c, seg_mode == 1 ? "up_seg_early" : "up_seg");
  if (seg_mode == 1) {
    ZQ_CUDA_TRY(cudaGetLastError());
    return ZQ_OK;
  }
  const unsigned wblocks = (unsigned)((c.m + kTopThreads / 32 - 1) / (kTopThreads / 32));
  time_begin(c, "up_top");
  if (rot) k_up_top_warp<T, true><<<wblocks, kTopThreads, 0, c.stream>>>(a, (int32_t)c.m);
  else k_up_top_warp<T, false><<<wblocks, kTopThreads, 0, c.stream>>>(a, (int32_t)c.m);
  time_begin(c, "up_top_block");
  if (rot) k_up_top<T, true><<<(unsigned)c.m, kTopThreads, 0, c.stream>>>(a);
  else k_up_top<T, false><<<(unsigned)c.m, kTopThreads, 0, c.stream>>>(a);
  time_end(c, "up_top_block");
  time_end(c, "up_top");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

template <typename T>
zq_status run_down(Ctx& c, const T* rec, T* xs, const T* w, T* out, const T* root_in, const double* rot) {
  SweepArgs<T> a = make_args<T>(c, rec, xs, w, out);
  a.root_in = root_in;
  a.rot = rot;
  const unsigned wblocks = (unsigned)((c.m + kTopThreads / 32 - 1) / (kTopThreads / 32));
  time_begin(c, "down_top");
  if (rot) k_down_top_warp<T, true><<<wblocks, kTopThreads, 0, c.stream>>>(a, (int32_t)c.m);
  else k_down_top_warp<T, false><<<wblocks, kTopThreads, 0, c.stream>>>(a, (int32_t)c.m);
  time_begin(c, "down_top_block");
  if (rot) k_down_top<T, true><<<(unsigned)c.m, kTopThreads, 0, c.stream>>>(a);
  else k_down_top<T, false><<<(unsigned)c.m, kTopThreads, 0, c.stream>>>(a);
  time_end(c, "down_top_block");
  time_end(c, "down_top");
  time_begin(c, "down_seg");
  if (rot) k_down_seg<T, true><<<c.num_sms * 16, kSegThreads, 0, c.stream>>>(a);
  else k_down_seg<T, false><<<c.num_sms * 16, kSegThreads, 0, c.stream>>>(a);
  time_end(c, "down_seg");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

}  // namespace

zq_status launch_apply_Q(Ctx& c, zq_prec prec, const void* v, int64_t /*ldv*/, void* out, void* root_out,
                         const double* rot, int seg_mode) {
  if (prec == ZQ_FP64)
    return run_up<double>(c, c.rec64, c.x64, static_cast<const double*>(v), static_cast<double*>(out),
                          static_cast<double*>(root_out), rot, seg_mode);
  return run_up<float>(c, c.rec32, c.x32, static_cast<const float*>(v), static_cast<float*>(out),
                       static_cast<float*>(root_out), rot, seg_mode);
}

zq_status launch_apply_QT(Ctx& c, zq_prec prec, const void* w, void* out, int64_t /*ldo*/, const void* root_in,
                          const double* rot) {
  if (prec == ZQ_FP64)
    return run_down<double>(c, c.rec64, c.x64, static_cast<const double*>(w), static_cast<double*>(out),
                            static_cast<const double*>(root_in), rot);
  return run_down<float>(c, c.rec32, c.x32, static_cast<const float*>(w), static_cast<float*>(out),
                         static_cast<const float*>(root_in), rot);
}

zq_status launch_apply_block(Ctx& c, bool up, zq_prec prec, int64_t k, const void* in, void* out) {
  if (prec == ZQ_TF32) return run_block_tc<Tf32, float>(c, up, (int32_t)k, in, out);
  if (prec == ZQ_BF16_TC) return run_block_tc<Bf16, __nv_bfloat16>(c, up, (int32_t)k, in, out);
  if (prec == ZQ_FP64) return run_block<double, double>(c, up, (int32_t)k, c.rec64, in, out);
  if (prec == ZQ_BF16) return run_block<__nv_bfloat16, float>(c, up, (int32_t)k, c.rec32, in, out);
  return run_block<float, float>(c, up, (int32_t)k, c.rec32, in, out);
}

}  // namespace zq
