// zq_scan.cu -- exclusive prefix sums of int32 (residue offsets, list
// compaction) and int64 (nonzero counts of the explicit Q~).  Up to 192 KB
// of values: one launch, one block.  Longer arrays: three
// launches (per-block totals, one block scanning the totals with a running
// carry, per-block scan plus carry).
#include "zq_internal.cuh"

namespace zq {

namespace {

constexpr int kThreads = 1024;
constexpr int kItems = 4;
constexpr int kTileN = kThreads * kItems;

template <typename I>
__device__ inline I warp_incl_scan(I v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    I t = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread over the block; returns the prefix
// and writes the block total to *total.
template <typename I>
__device__ inline I block_excl_scan(I v, I* sh, I* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  I inc = warp_incl_scan(v);
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    I w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
    I wi = warp_incl_scan(w);
    sh[lane] = wi - w;
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  I r = inc - v + sh[warp];
  *total = sh[32];
  __syncthreads();
  return r;
}

template <typename I>
__global__ void k_block_totals(const I* __restrict__ in, int64_t n, I* __restrict__ tot) {
  __shared__ I sh[33];
  int64_t base = (int64_t)blockIdx.x * kTileN + (int64_t)threadIdx.x * kItems;
  I s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i)
    if (base + i < n) s += in[base + i];
  I t;
  block_excl_scan(s, sh, &t);
  if (threadIdx.x == 0) tot[blockIdx.x] = t;
}

template <typename I>
__global__ void k_scan_totals(I* __restrict__ tot, int64_t nb, I* __restrict__ total) {
  __shared__ I sh[33];
  I carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    int64_t i = b0 + threadIdx.x;
    I v = (i < nb) ? tot[i] : 0;
    I t;
    I e = block_excl_scan(v, sh, &t);
    if (i < nb) tot[i] = carry + e;
    carry += t;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <typename I>
__global__ void k_block_scan(const I* __restrict__ in, int64_t n, const I* __restrict__ tot, I* __restrict__ out) {
  __shared__ I sh[33];
  int64_t base = (int64_t)blockIdx.x * kTileN + (int64_t)threadIdx.x * kItems;
  I v[kItems];
  I s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  I t;
  I e = block_excl_scan(s, sh, &t) + tot[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    if (base + i < n) out[base + i] = e;
    e += v[i];
  }
}

// Arrays of at most one_block_max<I>() values: one block.  The array is loaded
// into shared memory with coalesced loads (all in flight at once), thread t
// scans its consecutive chunk there, a block scan of the chunk sums gives
// the chunk prefixes, and the result goes out with coalesced stores.
constexpr int kOneBlockBytes = 192 * 1024;
template <typename I>
constexpr int64_t one_block_max() { return kOneBlockBytes / (int64_t)sizeof(I); }

template <typename I>
__global__ void __launch_bounds__(kThreads) k_scan_one_block(const I* in, int64_t n, I* out, I* total) {
  extern __shared__ __align__(16) unsigned char scan_smem[];
  I* v = reinterpret_cast<I*>(scan_smem);
  __shared__ I sh[33];
  for (int64_t i = threadIdx.x; i < n; i += kThreads) v[i] = in[i];
  __syncthreads();
  const int64_t per = (n + kThreads - 1) / kThreads;
  const int64_t b0 = (int64_t)threadIdx.x * per;
  const int64_t b1 = b0 + per < n ? b0 + per : n;
  I s = 0;
  for (int64_t i = b0; i < b1; ++i) s += v[i];
  I t;
  I run = block_excl_scan(s, sh, &t);  // ends with a barrier: every chunk sum is taken
  for (int64_t i = b0; i < b1; ++i) {
    const I x = v[i];
    v[i] = run;
    run += x;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += kThreads) out[i] = v[i];
  if (threadIdx.x == 0 && total) *total = t;
}

}  // namespace

int64_t scan_tmp_words(int64_t n) { return (n + kTileN - 1) / kTileN + 1; }

template <typename I>
zq_status scan_impl(Ctx& c, const I* in, I* out, int64_t n, I* tmp, I* total) {
  cudaStream_t s = c.stream;
  if (n <= 0) {
    if (total) ZQ_CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(I), s));
    return ZQ_OK;
  }
  if (n <= one_block_max<I>()) {
    const int smem = (int)(n * (int64_t)sizeof(I));
    if (smem > 48 * 1024)
      ZQ_CUDA_TRY(cudaFuncSetAttribute(k_scan_one_block<I>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOneBlockBytes));
    time_begin(c, "scan");
    k_scan_one_block<I><<<1, kThreads, smem, s>>>(in, n, out, total);
    time_end(c, "scan");
    ZQ_CUDA_TRY(cudaGetLastError());
    return ZQ_OK;
  }
  int64_t nb = (n + kTileN - 1) / kTileN;
  time_begin(c, "scan");
  k_block_totals<I><<<(unsigned)nb, kThreads, 0, s>>>(in, n, tmp);
  time_end(c, "scan");
  time_begin(c, "scan");
  k_scan_totals<I><<<1, kThreads, 0, s>>>(tmp, nb, total);
  time_end(c, "scan");
  time_begin(c, "scan");
  k_block_scan<I><<<(unsigned)nb, kThreads, 0, s>>>(in, n, tmp, out);
  time_end(c, "scan");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

// out[i] = sum_{k<i} in[k]; *total (device, may be NULL) = sum of all.
// in and out may alias.  tmp: scan_tmp_words(n) values of device scratch.
zq_status launch_exclusive_scan(Ctx& c, const int32_t* in, int32_t* out, int64_t n, int32_t* tmp,
                                int32_t* total) {
  return scan_impl<int32_t>(c, in, out, n, tmp, total);
}

zq_status launch_exclusive_scan64(Ctx& c, const int64_t* in, int64_t* out, int64_t n, int64_t* tmp,
                                  int64_t* total) {
  return scan_impl<int64_t>(c, in, out, n, tmp, total);
}

}  // namespace zq
