// Bead planes between the caller's order and the tree's sorted-position
// order.  The bisection of Sec. 2.1 orders each body's beads; the sweeps of
// Algorithms 2 and 3 visit them in that order, so a plane in that order is
// read (upward) or written (downward) in contiguous runs.  zq_pipeline uses
// these two passes around its sweeps: the gather into tree order runs on a
// side stream next to the transform build and also writes the inverse
// permutation; the pass back after the downward sweep is a gather too
// (coalesced writes in the caller's order, reads from the tree-ordered
// plane the sweep has just written, which is still in L2), instead of a
// scatter of 4-byte writes to random beads.
//
// Entry s of a tree-ordered plane is the caller's bead perm[s]; perm is a
// permutation of [0, N) (each body's range onto itself), written by the tree
// build, so every index below stays inside the N-entry planes, and
// iperm[perm[s]] = s is a permutation too.
#include "zq_internal.cuh"

namespace zq {
namespace {

constexpr int kOrderPassThreads = 256;
constexpr int kOrderPassBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kOrderPassThreads)
    k_to_tree(int64_t N, const int32_t* __restrict__ perm, const T* __restrict__ v, T* __restrict__ vt,
              int32_t* __restrict__ iperm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += stride) {
    const int64_t b = perm[s];
    iperm[b] = (int32_t)s;
    vt[s] = v[b];
    vt[N + s] = v[N + b];
    vt[2 * N + s] = v[2 * N + b];
  }
}

template <typename T>
__global__ void __launch_bounds__(kOrderPassThreads)
    k_from_tree(int64_t N, const int32_t* __restrict__ iperm, const T* __restrict__ ut, T* __restrict__ u) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < N; b += stride) {
    const int64_t s = iperm[b];
    u[b] = ut[s];
    u[N + b] = ut[N + s];
    u[2 * N + b] = ut[2 * N + s];
  }
}

unsigned order_grid(const Ctx& c) {
  const int64_t need = (c.N + kOrderPassThreads - 1) / kOrderPassThreads;
  const int64_t cap = (int64_t)c.num_sms * kOrderPassBlocksPerSM;
  return (unsigned)(need < cap ? need : cap);
}

}  // namespace

zq_status launch_to_tree(Ctx& c, zq_prec prec, const void* v, void* vt, int32_t* iperm) {
  if (c.N == 0) return ZQ_OK;
  time_begin(c, "to_tree");
  if (prec == ZQ_FP64)
    k_to_tree<double><<<order_grid(c), kOrderPassThreads, 0, c.stream>>>(
        c.N, c.perm, static_cast<const double*>(v), static_cast<double*>(vt), iperm);
  else
    k_to_tree<float><<<order_grid(c), kOrderPassThreads, 0, c.stream>>>(
        c.N, c.perm, static_cast<const float*>(v), static_cast<float*>(vt), iperm);
  time_end(c, "to_tree");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

zq_status launch_from_tree(Ctx& c, zq_prec prec, const void* ut, void* u, const int32_t* iperm) {
  if (c.N == 0) return ZQ_OK;
  time_begin(c, "from_tree");
  if (prec == ZQ_FP64)
    k_from_tree<double><<<order_grid(c), kOrderPassThreads, 0, c.stream>>>(
        c.N, iperm, static_cast<const double*>(ut), static_cast<double*>(u));
  else
    k_from_tree<float><<<order_grid(c), kOrderPassThreads, 0, c.stream>>>(
        c.N, iperm, static_cast<const float*>(ut), static_cast<float*>(u));
  time_end(c, "from_tree");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

}  // namespace zq
