// zq_sort.cu -- per-body sort of the bisection keys, ties broken by the
// body-local bead index (Sec. 2.1 readings: beads sharing a 21-bit cell are
// separated by their index bits).
//
// Bodies above kSmallSortMax beads (smaller ones are sorted inside the
// per-body tree kernel, zq_smalltree.cu): stable LSD radix sort, 4 passes
// of 8 bits over the high 32 key bits (the first 10 2/3 octree levels);
// stability keeps equal keys in bead (= index) order.  Then the runs of
// beads that share their high 32 bits are sorted by the low bits: runs of
// at most 32 by insertion, one thread each (k_sort_fixup); longer ones,
// listed by the fix-up, by one thread block each with a stable LSD radix
// sort over the low 32 bits in global memory (k_sort_runs), which takes any
// run length and does nothing when no run is listed.
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

// Runs of equal high key halves in a body's sorted keys [0, n): each run
// start p of length 2..32 is insertion-sorted by the full key (stable: the
// run is in index order); longer runs are listed for k_sort_runs (start,
// length; the end found by binary search on the sorted high halves).
constexpr int kFixupMax = 32;

__global__ void k_sort_fixup(uint64_t* __restrict__ key, int32_t* __restrict__ val, int64_t n,
                             int2* __restrict__ runs, int32_t* __restrict__ nruns) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const uint32_t hk = (uint32_t)(key[p] >> 32);
  if (p > 0 && (uint32_t)(key[p - 1] >> 32) == hk) return;  // not a run start
  int64_t L = 1;
  while (p + L < n && L <= kFixupMax && (uint32_t)(key[p + L] >> 32) == hk) ++L;
  if (L == 1) return;
  if (L > kFixupMax) {
    int64_t lo = p + L, hi = n;  // first position past the run
    while (lo < hi) {
      const int64_t md = (lo + hi) >> 1;
      if ((uint32_t)(key[md] >> 32) == hk) lo = md + 1; else hi = md;
    }
    const int32_t slot = atomicAdd(nruns, 1);
    runs[slot] = make_int2((int32_t)p, (int32_t)(lo - p));
    return;
  }
  for (int64_t u = p + 1; u < p + L; ++u) {
    const uint64_t k = key[u];
    const int32_t v = val[u];
    int64_t w = u - 1;
    while (w >= p && key[w] > k) {
      key[w + 1] = key[w];
      val[w + 1] = val[w];
      --w;
    }
    key[w + 1] = k;
    val[w + 1] = v;
  }
}

// The listed long runs, one block per run: four stable LSD passes of 8 bits
// over the low key half, in global memory between the run and the same
// range of the scratch (tmpk, tmpv), a tile of blockDim keys at a time in
// order (ranks within a warp by digit_peers, then warp by warp), so equal
// digits keep their order.
constexpr int kRunThreads = 1024;
constexpr int kRunWarps = kRunThreads / 32;

__global__ void __launch_bounds__(kRunThreads)
k_sort_runs(uint64_t* __restrict__ key, int32_t* __restrict__ val, uint64_t* __restrict__ tmpk,
            int32_t* __restrict__ tmpv, const int2* __restrict__ runs, const int32_t* __restrict__ nruns) {
  __shared__ int32_t start[kDigits];
  __shared__ int32_t wc[kRunWarps][kDigits];
  const int nr = *nruns;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = blockIdx.x; r < nr; r += gridDim.x) {
    const int2 run = runs[r];
    const int64_t p = run.x, L = run.y;
    uint64_t* kin = key + p;
    int32_t* vin = val + p;
    uint64_t* kout = tmpk + p;
    int32_t* vout = tmpv + p;
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 8 * pass;
      for (int d = threadIdx.x; d < kDigits; d += blockDim.x) start[d] = 0;
      __syncthreads();
      for (int64_t i = threadIdx.x; i < L; i += blockDim.x) atomicAdd(&start[(kin[i] >> shift) & (kDigits - 1)], 1);
      __syncthreads();
      if (threadIdx.x < 32) {  // exclusive scan of the digit counts, 8 per lane
        constexpr int kPer = kDigits / 32;
        int32_t v[kPer], t = 0;
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
          v[e] = start[lane * kPer + e];
          t += v[e];
        }
        int32_t inc = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t q = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += q;
        }
        int32_t run_ = inc - t;
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
          start[lane * kPer + e] = run_;
          run_ += v[e];
        }
      }
      __syncthreads();
      for (int64_t base = 0; base < L; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < L;
        uint64_t k = 0;
        int32_t v = 0;
        int dg = kDigits + lane;
        if (ok) {
          k = kin[i];
          v = vin[i];
          dg = (int)((k >> shift) & (kDigits - 1));
        }
        for (int d = lane; d < kDigits; d += 32) wc[warp][d] = 0;
        __syncwarp();
        const unsigned peers = digit_peers(dg, ok);
        if (ok && (peers & lt) == 0) wc[warp][dg] = __popc(peers);
        __syncthreads();
        for (int d = threadIdx.x; d < kDigits; d += blockDim.x) {  // warp-by-warp offsets of digit d
          int32_t run_ = start[d];
          for (int w = 0; w < kRunWarps; ++w) {
            const int32_t c = wc[w][d];
            wc[w][d] = run_;
            run_ += c;
          }
          start[d] = run_;
        }
        __syncthreads();
        if (ok) {
          const int32_t pos = wc[warp][dg] + __popc(peers & lt);
          kout[pos] = k;
          vout[pos] = v;
        }
        __syncthreads();
      }
      uint64_t* tk = kin; kin = kout; kout = tk;
      int32_t* tv = vin; vin = vout; vout = tv;
      __syncthreads();
    }
    // four passes: the sorted run is back in key / val
  }
}

}  // namespace

// The histogram and its scan scratch, then 2 words of run count (aligned),
// then the long-run list (an int2 per possible run start).
int64_t sort_hist_words(int64_t n_max) {
  const int64_t nblk = (n_max + kTile - 1) / kTile;
  const int64_t w = kDigits * nblk + scan_tmp_words(kDigits * nblk);
  return ((w + 1) & ~(int64_t)1) + 2 + 2 * (n_max + 1);
}

zq_status launch_sort(Ctx& c) {
  cudaStream_t s = c.stream;
  for (int32_t j : c.big_bodies) {
    int64_t o = c.off_h[j], n = c.off_h[j + 1] - o;
    int64_t nblk = (n + kTile - 1) / kTile;
    int32_t* hist = c.sort_hist;
    int32_t* tmp = c.sort_hist + kDigits * nblk;
    for (int pass = 4; pass < 8; ++pass) {  // the high 32 key bits
      const uint64_t* kin;
      const int32_t* vin;
      uint64_t* kout;
      int32_t* vout;
      if (pass == 4) {
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
    // runs of equal high halves, sorted by the low bits (the list of long
    // runs and its count live after the histogram in the sort scratch)
    int2* runs = reinterpret_cast<int2*>(c.sort_hist + sort_hist_words(n) - 2 * (n + 1));
    int32_t* nruns = c.sort_hist + sort_hist_words(n) - 2 * (n + 1) - 2;
    ZQ_CUDA_TRY(cudaMemsetAsync(nruns, 0, sizeof(int32_t), s));
    time_begin(c, "sort_fixup");
    k_sort_fixup<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.skey + o, c.perm + o, n, runs, nruns);
    time_end(c, "sort_fixup");
    time_begin(c, "sort_runs");
    k_sort_runs<<<(unsigned)c.num_sms, kRunThreads, 0, s>>>(c.skey + o, c.perm + o, c.key_tmp + o, c.perm_tmp + o,
                                                          runs, nruns);
    time_end(c, "sort_runs");
    ZQ_CUDA_TRY(cudaGetLastError());
  }
  return ZQ_OK;
}

}  // namespace zq
