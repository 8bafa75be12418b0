// zq_fused.cu -- the whole step of zq_pipeline after the tree, one body per
// thread block in one persistent launch.
//
// Bodies are independent (Q~ is block diagonal over the bodies, Sec. 1), so
// each body's node transforms (Sec. 3, Eq. 3.5, Case I of Eqs. 3.9-3.10),
// its upward sweep Q~ v (Algorithm 2, Eqs. 4.2-4.3) and its downward sweep
// Q~^T w (Algorithm 3, Theorem 4.3) can run to completion in one thread
// block without waiting for any other body.  The bodies are dealt to the
// thread blocks largest first, each to the block with the fewest nodes so
// far (longest processing time first, on the host at plan time).  A block
// takes its bodies in groups of at most kFusedMaxNodes nodes, sorts the
// group's nodes by (height, type) in shared memory, then:
//   heights 1, 2, ...: each node's transform (the node code of
//     zq_build_node.cuh, the same arithmetic as the level build) and, right
//     after it, the node's upward step from its children's Info-sets;
//   heights H, H - 1, ...: each node's downward step, from its Velocity-set
//     to its children's (each body root's is 0).
// One barrier per height.  There is no schedule across bodies: no level
// launches, no segment or bucket schedule, no tree-order passes; bead
// vectors are read and written through the tree's permutation directly.
//
// Layout: node state (centroid, T22) and the Info-/Velocity-sets by node
// id; records by node id at a fixed stride of kRecMax words (the products
// of this step read them back in the same launch, from L2).  The separate
// products (zq_apply_Q, ...) use a different record layout, so after a fused
// step the context holds no transforms for them until zq_build_transforms.
//
// Values written in this launch are read back only with coherent loads
// (plain or .cg), never through the read-only path.
#include "zq_build_node.cuh"
#include "zq_internal.cuh"
#include "zq_node.cuh"
#include "zq_real.cuh"

namespace zq {

namespace {

#ifndef ZQ_FUSED_THREADS
#define ZQ_FUSED_THREADS 128
#endif
constexpr int kFusedThreads = ZQ_FUSED_THREADS;
// nodes are sorted by (height, type), type = internal children (0, 1, 2),
// so that a warp mostly runs one kind of node transform
constexpr int kFusedBins = 3 * (kMaxHeight + 2);
constexpr int kFusedMaxNodes = kSmallSortMax - 1;  // nodes of one group; bodies of at most kSmallSortMax beads

template <typename T>
struct FusedArgs {
  BuildArgs b;           // coordinates, perm, counts and state by node id, records
  const int64_t* off;
  const int32_t* cl;
  const int32_t* cr;
  const int32_t* roff;
  const uint8_t* height;
  const int32_t* bin_start;   // [bins + 1]: the bodies of block b are bin_bodies[bin_start[b] ..]
  const int32_t* bin_bodies;
  const int32_t* root;        // root node id of every body
  int32_t m;
  int64_t N;
  bool tree_order;       // bead planes indexed by sorted position, not by bead
  const T* v;            // bead planes (3 x N) or null
  T* qv;                 // residues (R)
  const T* w;            // residues (R) or null
  T* qtw;                // bead planes (3 x N)
  T* xs;                 // Info-/Velocity-sets, 6 per node id
  const T* rec;          // the records this launch writes (b.rec32 or b.rec64)
};

template <typename T>
__device__ __forceinline__ void ld6(const T* p, T* v) {
#pragma unroll
  for (int i = 0; i < 6; ++i) v[i] = __ldcg(p + i);
}

template <typename T>
__device__ __forceinline__ void st6(T* p, const T* v) {
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = v[i];
}

template <typename T>
__device__ __forceinline__ int64_t bead_index(const FusedArgs<T>& a, int32_t code) {
  const int64_t pos = leaf_pos(code);
  return a.tree_order ? pos : (int64_t)a.b.perm[pos];
}

// Upward step of node q (its record was just written by this thread).
template <typename T>
__device__ __forceinline__ void up_step(const FusedArgs<T>& a, int64_t q, int2 cc, int type) {
  T X[6], Y[6], P[6];
  if (cc.x >= 0) {
    ld6(a.xs + 6 * (int64_t)cc.x, X);
  } else {
    const int64_t b = bead_index(a, cc.x);
    X[0] = a.v[b]; X[1] = a.v[a.N + b]; X[2] = a.v[2 * a.N + b];
  }
  if (cc.y >= 0) {
    ld6(a.xs + 6 * (int64_t)cc.y, Y);
  } else {
    const int64_t b = bead_index(a, cc.y);
    Y[0] = a.v[b]; Y[1] = a.v[a.N + b]; Y[2] = a.v[2 * a.N + b];
  }
  const T* r = a.rec + q * kRecMax;
  T* res = a.qv + a.roff[q];
  if (type == 0) up_node<T, 0, kLdCG>(r, X, Y, false, P, res);
  else if (type == 1) up_node<T, 1, kLdCG>(r, X, Y, cc.x >= 0, P, res);
  else up_node<T, 2, kLdCG>(r, X, Y, true, P, res);
  st6(a.xs + 6 * q, P);
}

// Downward step of node q: its Velocity-set (0 at the root) to its
// children's, or to the bead velocities of leaf children.
template <typename T>
__device__ __forceinline__ void down_step(const FusedArgs<T>& a, int64_t q, int2 cc, int type, bool root) {
  T Lp[6], Lx[6], Ly[6];
  if (root) {
#pragma unroll
    for (int i = 0; i < 6; ++i) Lp[i] = T(0);
  } else {
    ld6(a.xs + 6 * q, Lp);
  }
  const T* r = a.rec + q * kRecMax;
  const T* w = a.w + a.roff[q];
  if (type == 0) down_node<T, 0, kLdCG>(r, Lp, w, false, Lx, Ly);
  else if (type == 1) down_node<T, 1, kLdCG>(r, Lp, w, cc.x >= 0, Lx, Ly);
  else down_node<T, 2, kLdCG>(r, Lp, w, true, Lx, Ly);
  const int32_t ch[2] = {cc.x, cc.y};
  const T* L[2] = {Lx, Ly};
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    if (ch[e] >= 0) {
      st6(a.xs + 6 * (int64_t)ch[e], L[e]);
    } else {
      const int64_t b = bead_index(a, ch[e]);
      a.qtw[b] = L[e][0];
      a.qtw[a.N + b] = L[e][1];
      a.qtw[2 * a.N + b] = L[e][2];
    }
  }
}

template <class R, typename T>
__global__ void __launch_bounds__(kFusedThreads) k_fused_step(FusedArgs<T> a) {
  __shared__ int32_t ids[kFusedMaxNodes];
  __shared__ int32_t hs[kFusedBins];    // first index of each (height, type) in ids
  __shared__ int32_t fill[kFusedBins];
  __shared__ int32_t hmax;
  const int32_t g0 = a.bin_start[blockIdx.x], g1 = a.bin_start[blockIdx.x + 1];
  // the block's bodies in groups of at most kFusedMaxNodes nodes, each
  // group's nodes processed together, height by height
  for (int32_t gb = g0; gb < g1;) {
    int32_t ge = gb, total = 0;
    while (ge < g1) {
      const int32_t j = a.bin_bodies[ge];
      const int32_t nn = (int32_t)(a.off[j + 1] - a.off[j]) - 1;
      if (ge > gb && total + nn > kFusedMaxNodes) break;
      total += nn;
      ++ge;
    }
    if (threadIdx.x == 0) hmax = 0;
    for (int h = threadIdx.x; h < kFusedBins; h += blockDim.x) fill[h] = 0;
    __syncthreads();
    // counting sort of the group's nodes by (height, type)
    for (int32_t e = gb; e < ge; ++e) {
      const int32_t j = a.bin_bodies[e];
      const int64_t q0 = a.off[j] - j;
      const int32_t nn = (int32_t)(a.off[j + 1] - a.off[j]) - 1;
      for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) {
        const int64_t q = q0 + t;
        const int h = a.height[q];
        atomicAdd(&fill[3 * h + (a.cl[q] >= 0) + (a.cr[q] >= 0)], 1);
        atomicMax(&hmax, h);
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the counts by the first warp
      constexpr int kPer = (kFusedBins + 31) / 32;
      const int lane = threadIdx.x, h0 = lane * kPer;
      int32_t cnt[kPer], tot = 0;
#pragma unroll
      for (int e = 0; e < kPer; ++e) {
        cnt[e] = h0 + e < kFusedBins ? fill[h0 + e] : 0;
        tot += cnt[e];
      }
      int32_t inc = tot;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += u;
      }
      int32_t run = inc - tot;
#pragma unroll
      for (int e = 0; e < kPer; ++e) {
        if (h0 + e < kFusedBins) {
          hs[h0 + e] = run;
          fill[h0 + e] = run;
        }
        run += cnt[e];
      }
    }
    __syncthreads();
    for (int32_t e = gb; e < ge; ++e) {
      const int32_t j = a.bin_bodies[e];
      const int64_t q0 = a.off[j] - j;
      const int32_t nn = (int32_t)(a.off[j + 1] - a.off[j]) - 1;
      for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) {
        const int64_t q = q0 + t;
        ids[atomicAdd(&fill[3 * a.height[q] + (a.cl[q] >= 0) + (a.cr[q] >= 0)], 1)] = (int32_t)q;
      }
    }
    __syncthreads();
    const int H = hmax;
    // upward: transforms, then Q~ v, height by height
    for (int h = 1; h <= H; ++h) {
      const int32_t k1 = h < H ? hs[3 * h + 3] : total;
      for (int32_t k = hs[3 * h] + threadIdx.x; k < k1; k += blockDim.x) {
        const int64_t q = ids[k];
        const int2 cc = make_int2(a.cl[q], a.cr[q]);
        const int type = (cc.x >= 0) + (cc.y >= 0);
        const int64_t rw = q * kRecMax;
        const int4 kids = kids_by_id(a.b, cc.x, cc.y);
        if (type == 0) node_case1<R>(a.b, q, kids, rw);
        else if (type == 1) node_hh6<R>(a.b, q, kids, rw);
        else node_hh9<R>(a.b, q, kids, rw);
        if (a.v) up_step(a, q, cc, type);
      }
      __syncthreads();
    }
    // downward: Q~^T w from each body's root, whose Velocity-set is 0
    if (a.w) {
      for (int32_t e = gb + (int32_t)threadIdx.x / 8; e < ge; e += (int32_t)blockDim.x / 8)
        if (threadIdx.x % 8 < 6) a.xs[6 * (int64_t)a.root[a.bin_bodies[e]] + threadIdx.x % 8] = T(0);
      __syncthreads();
      for (int h = H; h >= 1; --h) {
        const int32_t k1 = h < H ? hs[3 * h + 3] : total;
        for (int32_t k = hs[3 * h] + threadIdx.x; k < k1; k += blockDim.x) {
          const int64_t q = ids[k];
          const int2 cc = make_int2(a.cl[q], a.cr[q]);
          down_step(a, q, cc, (cc.x >= 0) + (cc.y >= 0), false);
        }
        __syncthreads();
      }
    }
    gb = ge;
  }
}

template <class R, typename T>
zq_status run_fused(Ctx& c, const FusedArgs<T>& a) {
  time_begin(c, "fused");
  k_fused_step<R, T><<<(unsigned)c.fused_bins, kFusedThreads, 0, c.stream>>>(a);
  time_end(c, "fused");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

}  // namespace

bool fused_step_possible(const Ctx& c) { return c.have_tree && c.big_bodies.empty() && c.fused_bins > 0; }

zq_status launch_fused_step(Ctx& c, zq_prec prec, const double* x, const double* y, const double* z,
                            const void* v, void* qv, const void* w, void* qtw) {
  if (!fused_step_possible(c)) return ZQ_ESTATE;
  BuildArgs b;
  b.x = x; b.y = y; b.z = z;
  b.off = c.off; b.perm = c.perm; b.sc = nullptr; b.cnt = c.cnt; b.sheight = nullptr; b.sid = nullptr;
  b.bstart = nullptr; b.srw = nullptr; b.cut = c.cut;
  b.ctab = c.count_tab;
  b.ctab2 = c.count_tab2;
  b.st = c.st64;
  b.rec64 = prec == ZQ_FP64 ? c.rec64 : nullptr;
  b.rec32 = prec == ZQ_FP64 ? nullptr : c.rec32;
  b.err = c.counters + 2;
  c.st_is_dd = c.build_dd;
  auto fill = [&](auto& a, auto* rec, auto* xs) {
    using T = std::remove_pointer_t<decltype(xs)>;
    a.b = b;
    a.off = c.off; a.cl = c.cl; a.cr = c.cr; a.roff = c.roff; a.height = c.height;
    a.bin_start = c.fused_bin_start; a.bin_bodies = c.fused_bin_bodies; a.root = c.root;
    a.m = (int32_t)c.m; a.N = c.N; a.tree_order = c.tree_order;
    a.v = static_cast<const T*>(v); a.qv = static_cast<T*>(qv);
    a.w = static_cast<const T*>(w); a.qtw = static_cast<T*>(qtw);
    a.xs = xs; a.rec = rec;
  };
  if (prec == ZQ_FP64) {
    FusedArgs<double> a;
    fill(a, c.rec64, c.x64);
    return c.build_dd ? run_fused<dd, double>(c, a) : run_fused<double, double>(c, a);
  }
  FusedArgs<float> a;
  fill(a, c.rec32, c.x32);
  return c.build_dd ? run_fused<dd, float>(c, a) : run_fused<double, float>(c, a);
}

}  // namespace zq
