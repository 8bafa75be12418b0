// zq_internal.cuh -- layout of the context and device helpers shared by the
// translation units of libzq.  Not part of the public ABI (include/zq.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "zq.h"

namespace zq {

// ----------------------------------------------------------------- limits
constexpr int kQBits = 21;            // bits per coordinate (Sec. 2.1 quantisation)
constexpr int kMaxHeight = 96;        // 63 coordinate + 32 index bisection levels + 1
constexpr int kSmallSortMax = 8192;   // bodies sorted inside one thread block
constexpr int64_t kMaxBeads = 700000000;  // N cap: node ids, positions and residue offsets fit int32
// Schedule: nodes of height 1..cut are processed level by level over all
// bodies at once, sorted by (height, type) into 3 * cut buckets (type 0:
// two leaf children, k = 3; 1: one, k = 6; 2: none, k = 9); the nodes
// above the cut ("tail") form one more bucket, processed one block per body.
constexpr int kDefaultCut = 15;
constexpr int kMaxCut = 21;           // 3 * 21 + 1 = 64 buckets
constexpr int kMaxBuckets = 3 * kMaxCut + 1;

// Sweeps work on segments: the maximal subtrees of at most kSegMax beads.
// The nodes of a segment keep the node-id range of its subtree (a subtree's
// split positions are contiguous) but are reordered inside it by height,
// so one thread block can sweep the segment height by height in shared
// memory.  Nodes above all segments ("top" nodes, more than kSegMax beads)
// keep position = node id and are swept one thread block per body.
#ifndef ZQ_SEG_MAX
#define ZQ_SEG_MAX 512
#endif
constexpr int kSegMax = ZQ_SEG_MAX;

// Node records (float or double words), compact and type-specific.  With
// A = M^T (k x 3) built from [T22_x | T22_y | K], K = sqrt(n_x n_y/n)[d]x,
// the Householder vectors of the LQ have structural zeros; only the
// possibly nonzero entries are stored (0-based row indices of A):
//   type 0 (k = 3, Case I), 12 words: [0] alpha [1] beta [2..10] G row-major
//   type 1 (k = 6: rows 0-2 T22 of the internal child, 3-5 K), 16 words:
//     [0] alpha [1] beta [2..4] tau_1..3 [5,6] v1(4,5) [7..9] v2(3,4,5)
//     [10..12] v3(3,4,5)
//   type 2 (k = 9: rows 0-2 T22_x, 3-5 T22_y, 6-8 K), 20 words:
//     [0] alpha [1] beta [2..4] tau [5..7] v1(3,7,8) [8..12] v2(3,4,6,7,8)
//     [13..18] v3(3..8)
// (v_j(j) = 1 implicit.)  Records are stored compactly in position order
// (segments, heights inside segments); prw[p] is the record offset of
// position p in units of 4 words (all record sizes are multiples of 4).
__host__ __device__ constexpr int rec_words(int type) { return type == 0 ? 12 : (type == 1 ? 16 : 20); }
constexpr int kRecMax = 20;
// Dense export layout (zq_get_records): 28 doubles per node.
constexpr int kRec = 28;
// FP64 build state per node: centroid (3), T22 packed lower (6), pad (1).
constexpr int kState = 10;

// sqrt(n) and 1/sqrt(n) for bead counts n < kCountTab (built once per context).
constexpr int kCountTab = 1 << 16;

// Device error word bits (reported by zq_sync).
constexpr int kErrNonFinite = 1;
constexpr int kErrDegenerate = 2;

struct AxisQuant;  // quantiser constants of one body and axis (below)

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // side streams forked from and joined back into `stream` with events (so
  // graph capture sees one DAG): 0..2 concurrent per-body tree launches
  // (0 also Q~^T w next to Q~ v), 3 host-to-device copies of the vectors
  cudaStream_t side[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int num_sms = 0;
  // sizes of the allocated buffers
  int64_t cap_N = 0, cap_m = 0;
  // current problem
  int64_t N = 0, m = 0, nodes = 0, R = 0;
  int cut = kDefaultCut;
  bool have_tree = false, have_xform = false, have64 = false, have32 = false;
  bool build_dd = true;    // build the transforms in double-single (else native FP64)
  bool tree_order = false; // bead vectors of the products are in tree (sorted-position) order
  bool fused_step = false; // zq_pipeline runs the step after the tree as one per-body launch
  bool have_sched = false; // the segment and bucket schedules of the current tree exist
  bool st_is_dd = false;   // representation of st64 written by the last build
  std::vector<int64_t> off_h;
  std::vector<int32_t> fused_bins_h;  // host copies (kept alive for their upload): starts, then bodies
  std::vector<int32_t> small_bodies;  // n_j <= kSmallSortMax, grouped by size class
  std::vector<int32_t> big_bodies;    // n_j > kSmallSortMax (device-wide tree kernels)
  int small_class_start[5] = {0, 0, 0, 0, 0};
  int32_t max_small = 0;
  // device buffers (bodies)
  int64_t* off = nullptr;        // [m+1]
  int32_t* small_d = nullptr;    // [m] ids of small bodies
  // fused step: the bodies dealt to fused_bins thread blocks, largest
  // first, each to the block with the fewest nodes so far (LPT)
  int32_t fused_bins = 0;
  int32_t* fused_bin_start = nullptr;   // [m + 1] (first fused_bins + 1 used)
  int32_t* fused_bin_bodies = nullptr;  // [m]
  int32_t* bead_body = nullptr;  // [N] body of each bead / sorted position
  uint64_t* aabb = nullptr;      // [m * 6] ordered-int encoded lo[3], hi[3]
  AxisQuant* body_q = nullptr;   // [m * 3] quantiser constants per axis (bodies above kSmallSortMax)
  double* count_tab = nullptr;   // [2 * kCountTab]: sqrt(n), 1/sqrt(n)
  float2* count_tab2 = nullptr;  // the same as double-single pairs
  int32_t* root = nullptr;       // [m] root node id
  // beads
  uint64_t* key = nullptr;       // [N] Morton keys in bead order
  uint64_t* skey = nullptr;      // [N] keys in sorted order
  int32_t* perm = nullptr;       // [N] sorted position -> bead index
  uint64_t* key_tmp = nullptr;   // [N] radix-sort ping-pong
  int32_t* perm_tmp = nullptr;   // [N]
  int32_t* sort_hist = nullptr;  // radix-sort histograms
  int64_t sort_hist_cap = 0;
  // internal nodes, id q = off[j] - j + split position
  uint8_t* lcp = nullptr;        // [nodes]
  int32_t* cl = nullptr;         // [nodes] child codes
  int32_t* cr = nullptr;
  int32_t* first = nullptr;      // [nodes] first sorted position
  int32_t* cnt = nullptr;        // [nodes] beads below
  uint8_t* height = nullptr;     // [nodes]
  int32_t* roff = nullptr;       // [nodes] residue offsets
  int32_t* scan_tmp = nullptr;   // [nodes + blocks] scan workspace
  int32_t* counters = nullptr;   // [4]: spare, spare, err, spare
  // schedule, indexed by slot (the processing order; see kDefaultCut)
  int32_t* sid = nullptr;        // [nodes] slot -> node id
  int32_t* slot_of = nullptr;    // [nodes] node id -> slot
  int4* sc = nullptr;            // [nodes] children: (x, y, n_x, n_y); x, y >= 0 child
                                 // slot, < 0 leaf: -1 - its bead's coordinate index
  uint8_t* sheight = nullptr;    // [nodes] height
  int32_t* bstart = nullptr;     // [kMaxBuckets + 1] first slot of each bucket
  int32_t* bhist = nullptr;      // bucket-sort histograms
  int64_t bhist_cap = 0;
  // segments (see kSegMax), by position p (node id order with each segment
  // reordered by height)
  int32_t* pos_of = nullptr;     // [nodes] node id -> position
  int32_t* pnode = nullptr;      // [nodes] position -> node id
  int2* pc = nullptr;            // [nodes] child codes: >= 0 child position, < 0 leaf
  int32_t* proff = nullptr;      // [nodes] residue offset
  uint8_t* ph = nullptr;         // [nodes] height
  int32_t* prw = nullptr;        // [nodes + 1] record offset (4-word units, read as uint32)
  int32_t* seg_r = nullptr;      // [nodes] per segment: residue offset of its first node (its
                                 // residues are [seg_r, seg_r + 3 (nodes - 1)), contiguous)
  int4* seg = nullptr;           // [nodes] per segment: first position, nodes, first sorted
                                 // bead, 1 if its root is a body root (first nseg used)
  int32_t* topv = nullptr;       // [nodes] top nodes (= positions) of body j at
                                 // [off[j] - j, off[j] - j + top_cnt[j]) (its node ids' range)
  int32_t* top_cnt = nullptr;    // [m] top nodes per body
  int32_t* nseg = nullptr;       // [2] device counts: segments, top nodes
  int32_t* srw = nullptr;        // [nodes] record offset of each build slot (4-word units)
  // transforms, by slot
  double* st64 = nullptr;        // [nodes * kState]
  double* rec64 = nullptr;       // [nodes * kRecMax] compact records, by position
  float* rec32 = nullptr;        // [nodes * kRecMax]
  // sweep scratch: Info-sets / Velocity-sets of segment roots and top nodes,
  // by position
  double* x64 = nullptr;         // [nodes * 6]
  float* x32 = nullptr;          // [nodes * 6]
  double* x64b = nullptr;        // second copies: Q~^T w on a side stream while
  float* x32b = nullptr;         // Q~ v runs on the context stream (zq_pipeline)
  // block form (k right-hand sides): Info-/Velocity-sets of every node
  void* xblk = nullptr;          // [nodes * 6 * k] of the arithmetic type
  int64_t xblk_bytes = 0;
  // staging for host-buffer calls (bytes)
  void* stage = nullptr;
  int64_t stage_cap = 0;
  // zq_pipeline's bead planes in tree order: v gathered for the upward
  // sweep, then Q~^T w before its scatter (bytes)
  void* ord = nullptr;
  int64_t ord_cap = 0;
  // a step captured as a CUDA graph (zq_pipeline with ZQ_GRAPH): replayed
  // while every argument and the plan generation are unchanged
  uint64_t plan_gen = 0;         // bumped whenever the launch plan or a buffer changes
  cudaGraphExec_t gexec = nullptr;
  std::vector<uintptr_t> gkey;
  int64_t glaunches = 0;         // kernels in the captured step
  // kernel timing hook
  char time_name[32] = {0};
  cudaEvent_t time_ev0 = nullptr, time_ev1 = nullptr;
  bool time_started = false;  // start recorded in the current API call
  int64_t launches = 0;       // kernels launched by this context
};

// Every kernel launch goes through time_begin / time_end: counts the launch
// and brackets it with the caller's events when it is the timed kernel.
// The records are external, so inside a captured step (ZQ_GRAPH) they become
// event-record nodes that time every replay.
inline void time_record(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
  else cudaEventRecord(ev, s);
}
inline void time_begin(Ctx& c, const char* name) {
  ++c.launches;
  if (c.time_ev0 && !c.time_started && __builtin_strcmp(c.time_name, name) == 0) {
    time_record(c.time_ev0, c.stream);
    c.time_started = true;
  }
}
// A bracket around several launches (no launch of its own).
inline void time_open(Ctx& c, const char* name) {
  if (c.time_ev0 && !c.time_started && __builtin_strcmp(c.time_name, name) == 0) {
    time_record(c.time_ev0, c.stream);
    c.time_started = true;
  }
}
inline void time_end(const Ctx& c, const char* name) {
  if (c.time_ev1 && __builtin_strcmp(c.time_name, name) == 0) time_record(c.time_ev1, c.stream);
}

// --------------------------------------------------------------- helpers
__host__ __device__ inline bool is_leaf(int32_t code) { return code < 0; }

// Lanes of the warp holding the same BITS-bit digit as this lane (v: this
// lane holds one; a lane without one gets only itself), from one ballot per
// digit bit: the stable ranking step of the radix sorts and the bucket
// schedule.  Measured about 1.7 times faster per sort pass than
// __match_any_sync on this GPU.
template <int BITS = 8>
__device__ __forceinline__ unsigned digit_peers(int dg, bool v) {
  unsigned m = __ballot_sync(0xffffffffu, v);
#pragma unroll
  for (int b = 0; b < BITS; ++b) {
    const bool bit = (dg >> b) & 1;
    const unsigned bb = __ballot_sync(0xffffffffu, bit);
    m &= bit ? bb : ~bb;
  }
  return v ? m : (1u << (threadIdx.x & 31));
}
__host__ __device__ inline int32_t leaf_pos(int32_t code) { return -1 - code; }

// Bucket of a node of height h and type t (see kDefaultCut).
__host__ __device__ inline int bucket_of(int h, int t, int cut) {
  return h <= cut ? 3 * (h - 1) + t : 3 * cut;
}

// Range [lo, hi) of slots in [a, b) whose node id lies in [ida, idb); the
// node ids of those slots increase with the slot.
__device__ inline void id_range(const int32_t* __restrict__ sid, int32_t a, int32_t b, int64_t ida,
                                int64_t idb, int32_t* lo, int32_t* hi) {
  int32_t l = a, r = b;
  while (l < r) { int32_t md = (l + r) >> 1; if (sid[md] < ida) l = md + 1; else r = md; }
  *lo = l;
  r = b;
  while (l < r) { int32_t md = (l + r) >> 1; if (sid[md] < idb) l = md + 1; else r = md; }
  *hi = l;
}

// Body of a global sorted position / bead index: largest j with off[j] <= i.
__device__ inline int32_t body_of_bead(const int64_t* __restrict__ off, int64_t m, int64_t i) {
  int64_t lo = 0, hi = m - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return (int32_t)lo;
}

// Block-local counting sort of up to kHeightSorted items by height (order
// within a height arbitrary).  item(t) -> (id, height) for t in [0, n).
// On return (true): ids[k] in height order, hs[h] = first k of height h
// (hs[h + 1] its end), lim = {lowest, highest height}.  n > kHeightSorted:
// returns false (lim still set) and the caller scans instead.  All threads
// of the block must call.
constexpr int kHeightSorted = 4096;
struct HeightSort {
  int32_t ids[kHeightSorted];
  int32_t hs[kMaxHeight + 2];
  int lim[2];
};

template <class Item>
__device__ bool sort_by_height(int32_t n, Item item, HeightSort& S) {
  __syncthreads();  // S may still be read from a previous use
  for (int h = threadIdx.x; h < kMaxHeight + 2; h += blockDim.x) S.hs[h] = 0;
  if (threadIdx.x == 0) {
    S.lim[0] = kMaxHeight + 1;
    S.lim[1] = 0;
  }
  __syncthreads();
  for (int32_t t = threadIdx.x; t < n; t += blockDim.x) {
    const int h = item(t).y;
    atomicAdd(&S.hs[h], 1);
    atomicMin(&S.lim[0], h);
    atomicMax(&S.lim[1], h);
  }
  __syncthreads();
  if (n > kHeightSorted) return false;
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int h = 0; h < kMaxHeight + 2; ++h) {
      const int32_t v = S.hs[h];
      S.hs[h] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int32_t t = threadIdx.x; t < n; t += blockDim.x) {
    const int2 it = item(t);
    S.ids[atomicAdd(&S.hs[it.y], 1)] = it.x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // hs[h] is now the end of height h: shift back
    for (int h = kMaxHeight + 1; h > 0; --h) S.hs[h] = S.hs[h - 1];
    S.hs[0] = 0;
  }
  __syncthreads();
  return true;
}

// Bisection keys (Sec. 2.1): q = floor((p - lo) / (hi - lo) * 2^21) per
// axis, clamped to 2^21 - 1, in FP64 with correctly rounded subtraction and
// division (the tree is bit-exact with the oracle's).
__device__ __forceinline__ uint32_t quantise_exact(double p, double lo, double hi) {
  if (!(hi > lo)) return 0u;
  const double t = __ddiv_rn(__dsub_rn(p, lo), __dsub_rn(hi, lo));
  const double s = floor(__dmul_rn(t, (double)(1u << kQBits)));
  const double top = (double)((1u << kQBits) - 1);
  return s >= top ? ((1u << kQBits) - 1) : (uint32_t)s;
}

// The quantiser's constants for one body and axis.  The scaled coordinate
// p s + c (s = 2^21 / (hi - lo), c = -lo s) is one FP64 fused multiply-add;
// it differs from 2^21 times quantise_exact's quotient by less than
//   2^21 (3 + 3) 2^-53 + |lo| s 2^-53
// (the roundings of hi - lo, s, c and the fused multiply-add, and of the
// exact formula's subtraction and division; the second term from c), so
// its floor is the exact formula's whenever it lies farther than
// B = 2^-27 + |lo| s 2^-51 (the bound with a factor of 4 to spare) from
// every integer.  beta is the exponent with B < 2^-beta; -1 marks a flat
// axis (every bead quantises to 0), 0 a body so small against its
// coordinates that only the exact formula is used.
struct AxisQuant {
  double s, c;
  int beta;
};

__device__ __forceinline__ AxisQuant axis_quant(double lo, double hi) {
  AxisQuant q;
  if (!(hi > lo)) {
    q.s = 0.0;
    q.c = 0.0;
    q.beta = -1;
    return q;
  }
  q.s = (double)(1u << kQBits) / (hi - lo);
  q.c = __dmul_rn(-lo, q.s);
  const double B = 0x1p-27 + fabs(lo) * q.s * 0x1p-51;
  const int beta = -(ilogb(B) + 1);
  q.beta = beta > 0 ? beta : 0;
  return q;
}

// quantise_exact(p, lo, hi) for a body whose axis is not flat (q.beta >=
// 0): the floor is read from the bits of p s + c (integer instructions
// only) unless that value lies within 2^-beta of an integer, is negative,
// or reaches the top cell; those beads take the exact formula.
__device__ __forceinline__ uint32_t quantise_fma(double p, const AxisQuant& q, double lo, double hi) {
  const double v = __fma_rn(p, q.s, q.c);
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const int beta = q.beta;
  if ((b >> 63) == 0 && beta > 0) {
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    if (e >= 0 && e <= 20) {
      // v = M 2^(e - 52): integer part and fraction in units of 2^(e - 52)
      const int fbits = 52 - e;
      const unsigned long long ip = M >> fbits;
      const unsigned long long fr = M & ((1ull << fbits) - 1);
      const unsigned long long margin = fbits > beta ? 1ull << (fbits - beta) : 1ull;
      if (fr > margin && fr < (1ull << fbits) - margin && ip < (1ull << kQBits) - 1) return (uint32_t)ip;
    } else if (e < 0 && e >= -beta) {
      // 2^-beta <= v < 1: the floor is 0 unless v is within 2^-beta of 1
      // (for v in [1/2, 1), v = M 2^-53)
      if (e <= -2 || (1ull << 53) - M >= (1ull << (53 - beta))) return 0u;
    }
  }
  return quantise_exact(p, lo, hi);
}

// Bit interleave: bit b of v to bit 3 b.
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t s = v & 0x1fffffull;
  s = (s | (s << 32)) & 0x1f00000000ffffull;
  s = (s | (s << 16)) & 0x1f0000ff0000ffull;
  s = (s | (s << 8)) & 0x100f00f00f00f00full;
  s = (s | (s << 4)) & 0x10c30c30c30c30c3ull;
  s = (s | (s << 2)) & 0x1249249249249249ull;
  return s;
}

// Key of a bead: z, then y, then x bit per octree level, most significant
// first (the bisection order of Sec. 2.1).
__device__ __forceinline__ uint64_t bead_key(uint32_t qx, uint32_t qy, uint32_t qz) {
  return spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
}

// Orderable unsigned encoding of a double (for atomicMin/Max).
__device__ inline unsigned long long ord_encode(double d) {
  unsigned long long u = (unsigned long long)__double_as_longlong(d);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ inline double ord_decode(unsigned long long u) {
  return __longlong_as_double((long long)((u >> 63) ? (u & 0x7fffffffffffffffull) : ~u));
}

#define ZQ_TRY_STATUS(expr)                       \
  do {                                            \
    zq_status _st = (expr);                       \
    if (_st != ZQ_OK) return _st;                 \
  } while (0)

#define ZQ_CUDA_TRY(expr)                         \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) return ZQ_ECUDA;       \
  } while (0)

// ---------------------------------------------------- launchers (per TU)
// zq_tree.cu
// the tree; with schedules, also the segment and bucket schedules that the
// level build and the separate sweeps need (launch_schedules)
zq_status launch_tree(Ctx& c, const double* x, const double* y, const double* z, bool schedules = true);
zq_status launch_schedules(Ctx& c);
zq_status launch_bead_body(Ctx& c);
// zq_smalltree.cu
int small_tree_class(int64_t n);
zq_status launch_small_trees(Ctx& c, const double* x, const double* y, const double* z);
zq_status launch_count_table(Ctx& c);
zq_status launch_count_table_dd(Ctx& c);
int64_t bucket_hist_words(int64_t nodes);
// zq_sort.cu
zq_status launch_sort(Ctx& c);
int64_t sort_hist_words(int64_t n_max);  // histogram + scan workspace of the largest body
// zq_scan.cu
zq_status launch_exclusive_scan(Ctx& c, const int32_t* in, int32_t* out, int64_t n, int32_t* tmp,
                                int32_t* total);
zq_status launch_exclusive_scan64(Ctx& c, const int64_t* in, int64_t* out, int64_t n, int64_t* tmp,
                                  int64_t* total);
int64_t scan_tmp_words(int64_t n);
// zq_qgen.cu: the explicit Q~ in CSR form (include/zq.h, zq_qgen)
zq_status launch_qgen_nnz(Ctx& c, int64_t* nnz_host);  // synchronises c.stream
zq_status launch_qgen(Ctx& c, zq_prec prec, int64_t* row_ptr, int32_t* col, void* val, void* uz);
// zq_seg.cu
zq_status launch_segments(Ctx& c);
// zq_build.cu
// which: bit 0 = FP64 records, bit 1 = FP32 records
// after_levels (may be empty): called once the launches of heights 1..cut
// are queued and before the nodes above the cut, so the caller can fork
// work that needs only those nodes (the segments whose root is at most at
// the cut) onto another stream.
zq_status launch_build(Ctx& c, const double* x, const double* y, const double* z, int which,
                       const std::function<zq_status()>& after_levels = {});
// zq_fused.cu: transforms, Q~ v and Q~^T w of every body in one launch
// (bodies of at most kSmallSortMax beads; records in the fused layout)
bool fused_step_possible(const Ctx& c);
zq_status launch_fused_step(Ctx& c, zq_prec prec, const double* x, const double* y, const double* z,
                            const void* v, void* qv, const void* w, void* qtw);
// zq_order.cu: bead planes (3 x N) to and from the tree's sorted-position
// order (entry s = bead perm[s]), on c.stream; launch_to_tree also writes
// the inverse permutation iperm[N], which launch_from_tree reads
zq_status launch_to_tree(Ctx& c, zq_prec prec, const void* v, void* vt, int32_t* iperm);
zq_status launch_from_tree(Ctx& c, zq_prec prec, const void* ut, void* u, const int32_t* iperm);
// zq_apply.cu
// root_out / root_in (6 m values, may be null): the root Info-set Q_Z v of
// every body / the root Velocity-set fed to Q~^T (null: zero).  rot (9 m
// FP64, may be null): per-body rotations R_j, the products taken with
// Q~ blockdiag(R_j^T) (bead vectors rotated by R_j^T in, R_j out).
// seg_mode: 0 = every segment and the top nodes; 1 = only the segments
// whose root height is at most the level cut (no top nodes); 2 = the other
// segments, then the top nodes (after a mode 1 launch)
zq_status launch_apply_Q(Ctx& c, zq_prec prec, const void* v, int64_t ldv, void* out,
                         void* root_out = nullptr, const double* rot = nullptr, int seg_mode = 0);
zq_status launch_apply_QT(Ctx& c, zq_prec prec, const void* w, void* out, int64_t ldo,
                          const void* root_in = nullptr, const double* rot = nullptr);
// up: out = Q~ V, else out = Q~^T W; rows of k values (see include/zq.h)
zq_status launch_apply_block(Ctx& c, bool up, zq_prec prec, int64_t k, const void* in, void* out);

}  // namespace zq
