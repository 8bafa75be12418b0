// zq_sort.cu -- per-body sort of the bisection keys, ties broken by the
// body-local bead index (Sec. 2.1 readings: beads sharing a 21-bit cell are
// separated by their index bits).
//
// Bodies above kSmallSortMax beads (smaller ones are sorted inside the
// per-body tree kernel, zq_smalltree.cu): stable LSD radix sort, 8 passes
// of 8 bits over the 64-bit key; stability keeps equal keys in bead (=
// index) order.
#include "zq_internal.cuh"

namespace zq {

namespace {

// ------------------------------------------------------------ radix (big)
// Eight passes of 8-bit digits.  A block owns a tile of kTile keys (kept in
// shared memory for the pass); warp w owns the w-th slice of the tile, in
// order.  Counting: per-block histogram.  Scatter: within a warp, lanes
// with the same digit are ranked by digit_peers in lane order, and
// the slices of a tile follow each other, so equal digits keep their input
// order (a stable pass); the global position of (digit, tile) comes from
// a scan of the per-tile histograms (digit-major).
constexpr int kRadixThreads = 256;
constexpr int kWarps = kRadixThreads / 32;
constexpr int kSlice = 128;                 // keys per warp
constexpr int kTile = kWarps * kSlice;      // 1024 keys per block
constexpr int kDigits = 256;

__global__ void __launch_bounds__(kRadixThreads)
k_radix_count(const uint64_t* __restrict__ kin, int64_t n, int shift, int32_t* __restrict__ hist,
              int64_t nblk) {
  __shared__ int32_t cnt[kDigits];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += kRadixThreads) {
    const int64_t e = base + i;
    if (e < n) atomicAdd(&cnt[(kin[e] >> shift) & (kDigits - 1)], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n,
                int64_t vbase, int shift, const int32_t* __restrict__ hist, int64_t nblk,
                uint64_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ uint64_t sk[kTile];
  __shared__ int32_t sv[kTile];
  __shared__ int32_t whist[kWarps][kDigits];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kTile;
  const int cnt = (int)(n - base < (int64_t)kTile ? n - base : (int64_t)kTile);
  for (int i = threadIdx.x; i < cnt; i += kRadixThreads) {
    sk[i] = kin[base + i];
    sv[i] = vin ? vin[base + i] : (int32_t)(vbase + base + i);
  }
  for (int d = lane; d < kDigits; d += 32) whist[warp][d] = 0;
  __syncthreads();
  const int c0 = min(cnt, warp * kSlice), c1 = min(cnt, c0 + kSlice);
  for (int b = c0; b < c1; b += 32) {
    const int i = b + lane;
    const bool v = i < c1;
    const int dg = v ? (int)((sk[i] >> shift) & (kDigits - 1)) : kDigits + lane;
    const unsigned peers = digit_peers(dg, v);
    if (v && (peers & lt) == 0) whist[warp][dg] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // thread d: first output position of (digit d, warp w) for every w
    const int d = threadIdx.x;
    int32_t run = hist[(int64_t)d * nblk + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const int32_t c = whist[w][d];
      whist[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int b = c0; b < c1; b += 32) {
    const int i = b + lane;
    const bool v = i < c1;
    uint64_t k = 0;
    int32_t val = 0;
    int dg = kDigits + lane;
    if (v) {
      k = sk[i];
      val = sv[i];
      dg = (int)((k >> shift) & (kDigits - 1));
    }
    const unsigned peers = digit_peers(dg, v);
    if (v) {
      const int32_t pos = whist[warp][dg] + __popc(peers & lt);
      kout[pos] = k;
      vout[pos] = val;
    }
    __syncwarp();
    if (v && (peers & lt) == 0) whist[warp][dg] += __popc(peers);
    __syncwarp();
  }
}

}  // namespace

int64_t sort_hist_words(int64_t n_max) {
  const int64_t nblk = (n_max + kTile - 1) / kTile;
  return kDigits * nblk + scan_tmp_words(kDigits * nblk);
}

zq_status launch_sort(Ctx& c) {
  cudaStream_t s = c.stream;
  for (int32_t j : c.big_bodies) {
    int64_t o = c.off_h[j], n = c.off_h[j + 1] - o;
    int64_t nblk = (n + kTile - 1) / kTile;
    int32_t* hist = c.sort_hist;
    int32_t* tmp = c.sort_hist + kDigits * nblk;
    for (int pass = 0; pass < 8; ++pass) {
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
      int shift = 8 * pass;
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
