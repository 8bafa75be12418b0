// zq_sort.cu -- per-body sort of the bisection keys, ties broken by the
// body-local bead index (Sec. 2.1 readings: beads sharing a 21-bit cell are
// separated by their index bits).
//
// Bodies above kSmallSortMax beads (smaller ones are sorted inside the
// per-body tree kernel, zq_smalltree.cu): stable LSD radix sort, 16 passes
// of 4 bits over the 64-bit key; stability keeps equal keys in bead (=
// index) order.
#include "zq_internal.cuh"

namespace zq {

namespace {

// ------------------------------------------------------------ radix (big)
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kDigits = 16;

__global__ void __launch_bounds__(kRadixThreads)
k_radix_count(const uint64_t* __restrict__ kin, int64_t n, int shift, int32_t* __restrict__ hist,
              int64_t nblk) {
  __shared__ int32_t cnt[kDigits];
  if (threadIdx.x < kDigits) cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)threadIdx.x * kRadixItems;
  for (int i = 0; i < kRadixItems; ++i) {
    int64_t e = base + i;
    if (e < n) atomicAdd(&cnt[(kin[e] >> shift) & (kDigits - 1)], 1);
  }
  __syncthreads();
  if (threadIdx.x < kDigits) hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

__device__ inline int32_t blk_excl(int32_t v, int32_t* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int32_t t = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += t;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int32_t w = (lane < (kRadixThreads >> 5)) ? sh[lane] : 0;
    int32_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int32_t t = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += t;
    }
    sh[lane] = wi - w;
  }
  __syncthreads();
  int32_t r = inc - v + sh[warp];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n,
                int64_t vbase, int shift, const int32_t* __restrict__ hist, int64_t nblk,
                uint64_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ int32_t sh[33];
  int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)threadIdx.x * kRadixItems;
  int32_t c[kDigits];
#pragma unroll
  for (int d = 0; d < kDigits; ++d) c[d] = 0;
  for (int i = 0; i < kRadixItems; ++i) {
    int64_t e = base + i;
    if (e < n) {
      int d = (int)((kin[e] >> shift) & (kDigits - 1));
#pragma unroll
      for (int dd = 0; dd < kDigits; ++dd) c[dd] += (dd == d);
    }
  }
  int32_t pos[kDigits];
#pragma unroll
  for (int d = 0; d < kDigits; ++d)
    pos[d] = blk_excl(c[d], sh) + hist[(int64_t)d * nblk + blockIdx.x];
  for (int i = 0; i < kRadixItems; ++i) {
    int64_t e = base + i;
    if (e < n) {
      uint64_t kk = kin[e];
      int d = (int)((kk >> shift) & (kDigits - 1));
      int32_t p = 0;
#pragma unroll
      for (int dd = 0; dd < kDigits; ++dd)
        if (dd == d) p = pos[dd]++;
      kout[p] = kk;
      vout[p] = vin ? vin[e] : (int32_t)(vbase + e);
    }
  }
}

}  // namespace

zq_status launch_sort(Ctx& c) {
  cudaStream_t s = c.stream;
  for (int32_t j : c.big_bodies) {
    int64_t o = c.off_h[j], n = c.off_h[j + 1] - o;
    int64_t nblk = (n + kRadixTile - 1) / kRadixTile;
    int32_t* hist = c.sort_hist;
    int32_t* tmp = c.sort_hist + kDigits * nblk;
    for (int pass = 0; pass < 16; ++pass) {
      const uint64_t* kin;
      const int32_t* vin;
      uint64_t* kout;
      int32_t* vout;
      if (pass == 0) {
        kin = c.key + o; vin = nullptr; kout = c.key_tmp + o; vout = c.perm_tmp + o;
      } else if (pass & 1) {
        kin = c.key_tmp + o; vin = c.perm_tmp + o; kout = c.skey + o; vout = c.perm + o;
      } else {
        kin = c.skey + o; vin = c.perm + o; kout = c.key_tmp + o; vout = c.perm_tmp + o;
      }
      int shift = 4 * pass;
      time_begin(c, "sort_radix_count");
      k_radix_count<<<(unsigned)nblk, kRadixThreads, 0, s>>>(kin, n, shift, hist, nblk);
      time_end(c, "sort_radix_count");
      zq_status st = launch_exclusive_scan(c, hist, hist, kDigits * nblk, tmp, nullptr);
      if (st != ZQ_OK) return st;
      time_begin(c, "sort_radix");
      k_radix_scatter<<<(unsigned)nblk, kRadixThreads, 0, s>>>(kin, vin, n, o, shift, hist, nblk,
                                                              kout, vout);
      time_end(c, "sort_radix");
      ZQ_CUDA_TRY(cudaGetLastError());
    }
  }
  return ZQ_OK;
}

}  // namespace zq
