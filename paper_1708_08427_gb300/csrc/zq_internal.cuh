// zq_internal.cuh -- layout of the context and device helpers shared by the
// translation units of libzq.  Not part of the public ABI (include/zq.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "zq.h"

namespace zq {

// ----------------------------------------------------------------- limits
constexpr int kQBits = 21;            // bits per coordinate (Sec. 2.1 quantisation)
constexpr int kMaxHeight = 96;        // 63 coordinate + 32 index bisection levels + 1
constexpr int kSmallSortMax = 8192;   // bodies sorted inside one thread block
constexpr int kDefaultTile = 2048;    // beads per sweep tile
constexpr int kMaxTile = 4096;      // FP64 sweep tile: 4096 * 50 B of shared memory

// Node record: one per internal node, float or double, kRec words.
//   [0] sqrt(n_x/n)  [1] sqrt(n_y/n)  [2..4] tau_1..tau_3 (Householder)
//   [5 ...] reflector tails v_1(2..k), v_2(3..k), v_3(4..k)  (k = 6, 9)
//   [5 .. 13] G row-major (k = 3, Case I)
// k = 3 + 3 * (number of internal children); the children are in the tree.
constexpr int kRec = 28;
// FP64 build state per node: centroid (3), T22 packed lower (6), pad (1).
constexpr int kState = 10;

// Device error word bits (reported by zq_sync).
constexpr int kErrNonFinite = 1;
constexpr int kErrDegenerate = 2;

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  // sizes of the allocated buffers
  int64_t cap_N = 0, cap_m = 0;
  // current problem
  int64_t N = 0, m = 0, nodes = 0, R = 0;
  int tile = kDefaultTile;
  bool have_tree = false, have_xform = false;
  std::vector<int64_t> off_h;
  std::vector<int32_t> small_bodies;  // n_j <= kSmallSortMax
  std::vector<int32_t> big_bodies;    // n_j > kSmallSortMax (device radix sort)
  std::vector<int32_t> top_bodies;    // n_j > tile (have nodes above the tiles)
  int32_t max_small = 0;
  // device buffers (bodies)
  int64_t* off = nullptr;        // [m+1]
  int32_t* small_d = nullptr;    // [m] ids of small bodies
  int32_t* top_d = nullptr;      // [m] ids of bodies with top nodes
  uint64_t* aabb = nullptr;      // [m * 6] ordered-int encoded lo[3], hi[3]
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
  int32_t* parent = nullptr;     // [nodes] (-1 at a body root)
  int32_t* flag = nullptr;       // [nodes] bottom-up arrival counters
  int32_t* roff = nullptr;       // [nodes] residue offsets
  int32_t* scan_tmp = nullptr;   // [nodes + blocks] scan workspace
  int32_t* tiles = nullptr;      // [nodes] tile-root ids
  int32_t* top = nullptr;        // [nodes] ids of nodes above the tiles
  int32_t* counters = nullptr;   // [4]: ntiles, ntop, err, spare
  // transforms
  double* st64 = nullptr;        // [nodes * kState]
  double* rec64 = nullptr;       // [nodes * kRec]
  float* rec32 = nullptr;        // [nodes * kRec]
  // sweep scratch: Info-sets / Velocity-sets of nodes outside the tiles
  double* x64 = nullptr;         // [nodes * 6]
  float* x32 = nullptr;          // [nodes * 6]
  // staging for host-buffer calls (bytes)
  void* stage = nullptr;
  int64_t stage_cap = 0;
  // kernel timing hook
  char time_name[32] = {0};
  cudaEvent_t time_ev0 = nullptr, time_ev1 = nullptr;
  int64_t launches = 0;  // kernels launched by this context
};

// Every kernel launch goes through time_begin / time_end: counts the launch
// and brackets it with the caller's events when it is the timed kernel.
inline void time_begin(Ctx& c, const char* name) {
  ++c.launches;
  if (c.time_ev0 && __builtin_strcmp(c.time_name, name) == 0) cudaEventRecord(c.time_ev0, c.stream);
}
inline void time_end(const Ctx& c, const char* name) {
  if (c.time_ev1 && __builtin_strcmp(c.time_name, name) == 0) cudaEventRecord(c.time_ev1, c.stream);
}

// --------------------------------------------------------------- helpers
__host__ __device__ inline bool is_leaf(int32_t code) { return code < 0; }
__host__ __device__ inline int32_t leaf_pos(int32_t code) { return -1 - code; }

// Body of a global sorted position / bead index: largest j with off[j] <= i.
__device__ inline int32_t body_of_bead(const int64_t* __restrict__ off, int64_t m, int64_t i) {
  int64_t lo = 0, hi = m - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return (int32_t)lo;
}

// Body of an internal node id: largest j with off[j] - j <= q.
__device__ inline int32_t body_of_node(const int64_t* __restrict__ off, int64_t m, int64_t q) {
  int64_t lo = 0, hi = m - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] - mid <= q) lo = mid; else hi = mid - 1;
  }
  return (int32_t)lo;
}

// Orderable unsigned encoding of a double (for atomicMin/Max).
__device__ inline unsigned long long ord_encode(double d) {
  unsigned long long u = (unsigned long long)__double_as_longlong(d);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ inline double ord_decode(unsigned long long u) {
  return __longlong_as_double((long long)((u >> 63) ? (u & 0x7fffffffffffffffull) : ~u));
}

#define ZQ_CUDA_TRY(expr)                         \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) return ZQ_ECUDA;       \
  } while (0)

// ---------------------------------------------------- launchers (per TU)
// zq_tree.cu
zq_status launch_tree(Ctx& c, const double* x, const double* y, const double* z);
// zq_sort.cu
zq_status launch_sort(Ctx& c);
// zq_scan.cu
zq_status launch_exclusive_scan(Ctx& c, const int32_t* in, int32_t* out, int64_t n, int32_t* tmp,
                                int32_t* total);
int64_t scan_tmp_words(int64_t n);
// zq_build.cu
zq_status launch_build(Ctx& c, const double* x, const double* y, const double* z);
// zq_apply.cu
zq_status launch_apply_Q(Ctx& c, zq_prec prec, const void* v, int64_t ldv, void* out);
zq_status launch_apply_QT(Ctx& c, zq_prec prec, const void* w, void* out, int64_t ldo);

}  // namespace zq
