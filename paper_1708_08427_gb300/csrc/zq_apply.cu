// zq_apply.cu -- the two sweeps.
//
// Upward (Q~ v, Algorithm 2, Eqs. 4.2-4.3): a leaf's Info-set is its bead
// vector f_i (Definition 4.1); for node p with children x, y
//   t_p = alpha t_x + beta t_y,   s = beta t_x - alpha t_y,
//   [r_p; eps_p] = G [r_x?; r_y?; s]   (r_c only for internal children),
// eps_p (k - 3 numbers) is p's Residue, written at its residue offset.
// Downward (Q~^T w, Algorithm 3, Theorem 4.3, Eqs. 4.6-4.7): the root
// Velocity-set is 0; for node p with Velocity-set [T; l] and residue
// coefficients w_p
//   [a_x?; a_y?; sigma] = G^T [l; w_p],
//   L_x = [alpha T + beta sigma; a_x],  L_y = [beta T - alpha sigma; a_y],
// and a leaf's velocity is the first three entries of its Velocity-set.
//
// G is applied as its three Householder reflectors (G u = H3 H2 H1 u,
// G^T z = H1 H2 H3 z), or as the explicit 3 x 3 matrix for Case I.
//
// Work split: one thread block per tile (a subtree of at most `tile`
// beads), level by level with the Info-/Velocity-sets in shared memory;
// nodes above the tiles are handled by one block per body, their sets in
// global scratch.  Upward: tiles, then tops.  Downward: tops, then tiles.
#include "zq_internal.cuh"

namespace zq {

namespace {

constexpr int kThreads = 256;

template <typename T>
struct ApplyArgs {
  const int64_t* off;
  int64_t m;
  int64_t N;
  const int32_t* perm;
  const int32_t* cl;
  const int32_t* cr;
  const int32_t* cnt;
  const int32_t* first;
  const int32_t* roff;
  const uint8_t* height;
  const int32_t* tiles;
  const int32_t* top;
  const int32_t* counters;
  const int32_t* top_bodies;
  const int32_t* root;
  const T* rec;
  T* xs;          // Info-/Velocity-sets of tile roots and top nodes [nodes * 6]
  const T* in;    // up: bead planes; down: residues
  T* out;         // up: residues; down: bead planes
};

// ---------------------------------------------------------- reflectors
// u <- H_j u for the reflector with tail v (entries j+1..K-1), v_j = 1.
template <typename T, int K, int J>
__device__ __forceinline__ void reflect(const T* __restrict__ rec, int tail, T tau, T (&u)[9]) {
  T w = u[J];
#pragma unroll
  for (int i = J + 1; i < K; ++i) w += rec[tail + i - J - 1] * u[i];
  w *= tau;
  u[J] -= w;
#pragma unroll
  for (int i = J + 1; i < K; ++i) u[i] -= w * rec[tail + i - J - 1];
}

template <typename T, int K>
__device__ __forceinline__ void g_apply(const T* __restrict__ rec, T (&u)[9]) {
  reflect<T, K, 0>(rec, 5, rec[2], u);
  reflect<T, K, 1>(rec, 5 + K - 1, rec[3], u);
  reflect<T, K, 2>(rec, 5 + 2 * K - 3, rec[4], u);
}

template <typename T, int K>
__device__ __forceinline__ void gt_apply(const T* __restrict__ rec, T (&u)[9]) {
  reflect<T, K, 2>(rec, 5 + 2 * K - 3, rec[4], u);
  reflect<T, K, 1>(rec, 5 + K - 1, rec[3], u);
  reflect<T, K, 0>(rec, 5, rec[2], u);
}

// ------------------------------------------------------------ node ops
// in: tx, ty (translational Info-sets), rx / ry (rotational, internal
// children only).  out: t, r; residues to res[0 .. k-4].
template <typename T>
__device__ __forceinline__ void up_node(const T* __restrict__ rec, bool xi, bool yi, const T* tx,
                                        const T* rx, const T* ty, const T* ry, T* t, T* r,
                                        T* __restrict__ res) {
  const T al = rec[0], be = rec[1];
  T u[9];
  int k = 0;
  if (xi) { u[0] = rx[0]; u[1] = rx[1]; u[2] = rx[2]; k = 3; }
  if (yi) { u[k] = ry[0]; u[k + 1] = ry[1]; u[k + 2] = ry[2]; k += 3; }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    t[a] = al * tx[a] + be * ty[a];
    u[k + a] = be * tx[a] - al * ty[a];
  }
  if (!xi && !yi) {
#pragma unroll
    for (int i = 0; i < 3; ++i) r[i] = rec[5 + 3 * i] * u[0] + rec[6 + 3 * i] * u[1] + rec[7 + 3 * i] * u[2];
    return;
  }
  if (xi && yi) {
    g_apply<T, 9>(rec, u);
#pragma unroll
    for (int i = 3; i < 9; ++i) res[i - 3] = u[i];
  } else {
    g_apply<T, 6>(rec, u);
#pragma unroll
    for (int i = 3; i < 6; ++i) res[i - 3] = u[i];
  }
  r[0] = u[0]; r[1] = u[1]; r[2] = u[2];
}

// in: Velocity-set Lp (6), residue coefficients w (k-3).  out: Lx, Ly (6
// each; entries 3..5 meaningful only for internal children).
template <typename T>
__device__ __forceinline__ void down_node(const T* __restrict__ rec, bool xi, bool yi, const T* Lp,
                                          const T* __restrict__ w, T* Lx, T* Ly) {
  const T al = rec[0], be = rec[1];
  T z[9];
  z[0] = Lp[3]; z[1] = Lp[4]; z[2] = Lp[5];
  T sg[3];
  if (!xi && !yi) {
#pragma unroll
    for (int j = 0; j < 3; ++j) sg[j] = rec[5 + j] * z[0] + rec[8 + j] * z[1] + rec[11 + j] * z[2];
  } else if (xi && yi) {
#pragma unroll
    for (int i = 3; i < 9; ++i) z[i] = w[i - 3];
    gt_apply<T, 9>(rec, z);
    Lx[3] = z[0]; Lx[4] = z[1]; Lx[5] = z[2];
    Ly[3] = z[3]; Ly[4] = z[4]; Ly[5] = z[5];
    sg[0] = z[6]; sg[1] = z[7]; sg[2] = z[8];
  } else {
#pragma unroll
    for (int i = 3; i < 6; ++i) z[i] = w[i - 3];
    gt_apply<T, 6>(rec, z);
    T* a = xi ? Lx : Ly;
    a[3] = z[0]; a[4] = z[1]; a[5] = z[2];
    sg[0] = z[3]; sg[1] = z[4]; sg[2] = z[5];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Lx[i] = al * Lp[i] + be * sg[i];
    Ly[i] = be * Lp[i] - al * sg[i];
  }
}

template <typename T>
__device__ __forceinline__ void load_rec(const T* __restrict__ g, T* r) {
#pragma unroll
  for (int i = 0; i < kRec; ++i) r[i] = __ldg(g + i);
}

template <typename T>
__device__ __forceinline__ void load_bead(const ApplyArgs<T>& a, int32_t code, T* t) {
  const int32_t i = a.perm[leaf_pos(code)];
  t[0] = a.in[i];
  t[1] = a.in[a.N + i];
  t[2] = a.in[2 * a.N + i];
}

template <typename T>
__device__ __forceinline__ void store_bead(const ApplyArgs<T>& a, int32_t code, const T* L) {
  const int32_t i = a.perm[leaf_pos(code)];
  a.out[i] = L[0];
  a.out[a.N + i] = L[1];
  a.out[2 * a.N + i] = L[2];
}

__device__ int make_levels(const uint8_t* __restrict__ hgt, int nn, uint16_t* list, int* lstart,
                           int* lcnt, int* hmax) {
  for (int i = threadIdx.x; i < kMaxHeight + 2; i += blockDim.x) lcnt[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < nn; i += blockDim.x) atomicAdd(&lcnt[hgt[i]], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0, H = 0;
    for (int h = 0; h <= kMaxHeight; ++h) {
      lstart[h] = s;
      s += lcnt[h];
      if (lcnt[h]) H = h;
      lcnt[h] = 0;
    }
    lstart[kMaxHeight + 1] = s;
    *hmax = H;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int h = hgt[i];
    list[lstart[h] + atomicAdd(&lcnt[h], 1)] = (uint16_t)i;
  }
  __syncthreads();
  return *hmax;
}

__device__ inline void top_range(const int32_t* top, int ntop, int64_t a, int64_t b, int* lo,
                                 int* hi) {
  int l = 0, r = ntop;
  while (l < r) { int md = (l + r) >> 1; if (top[md] < a) l = md + 1; else r = md; }
  *lo = l;
  r = ntop;
  while (l < r) { int md = (l + r) >> 1; if (top[md] < b) l = md + 1; else r = md; }
  *hi = l;
}

// -------------------------------------------------------------- upward
template <typename T>
__global__ void __launch_bounds__(kThreads) k_up_tiles(ApplyArgs<T> a, int tile) {
  extern __shared__ unsigned char smem_raw[];
  T* info = reinterpret_cast<T*>(smem_raw);
  uint16_t* list = reinterpret_cast<uint16_t*>(info + (size_t)tile * 6);
  __shared__ int lstart[kMaxHeight + 2], lcnt[kMaxHeight + 2], hmax;
  const int ntiles = a.counters[0];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int32_t R = a.tiles[t];
    const int32_t j = body_of_node(a.off, a.m, R);
    const int64_t base = (int64_t)a.first[R] - j;
    const int nn = a.cnt[R] - 1;
    const int H = make_levels(a.height + base, nn, list, lstart, lcnt, &hmax);
    for (int h = 1; h <= H; ++h) {
      for (int p = lstart[h] + threadIdx.x; p < lstart[h + 1]; p += blockDim.x) {
        const int li = list[p];
        const int64_t q = base + li;
        const int32_t lc = a.cl[q], rc = a.cr[q];
        T rec[kRec];
        load_rec(a.rec + q * kRec, rec);
        T bx[3], by[3];
        const T *tx, *rx = nullptr, *ty, *ry = nullptr;
        if (is_leaf(lc)) { load_bead(a, lc, bx); tx = bx; }
        else { tx = info + (lc - base) * 6; rx = tx + 3; }
        if (is_leaf(rc)) { load_bead(a, rc, by); ty = by; }
        else { ty = info + (rc - base) * 6; ry = ty + 3; }
        T tr[6];
        up_node(rec, !is_leaf(lc), !is_leaf(rc), tx, rx, ty, ry, tr, tr + 3, a.out + a.roff[q]);
        T* dst = info + (int64_t)li * 6;
#pragma unroll
        for (int i = 0; i < 6; ++i) dst[i] = tr[i];
      }
      __syncthreads();
    }
    const int64_t n_body = a.off[j + 1] - a.off[j];
    if (a.cnt[R] < n_body && threadIdx.x < 6)
      a.xs[(int64_t)R * 6 + threadIdx.x] = info[(R - base) * 6 + threadIdx.x];
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_up_top(ApplyArgs<T> a) {
  const int32_t j = a.top_bodies[blockIdx.x];
  const int64_t nb = a.off[j] - j, ne = a.off[j + 1] - (j + 1);
  int lo, hi;
  top_range(a.top, a.counters[1], nb, ne, &lo, &hi);
  const int H = a.height[a.root[j]];
  for (int h = 1; h <= H; ++h) {
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
      const int32_t q = a.top[p];
      if (a.height[q] != h) continue;
      const int32_t lc = a.cl[q], rc = a.cr[q];
      T rec[kRec];
      load_rec(a.rec + (int64_t)q * kRec, rec);
      T X[6], Y[6];
      if (is_leaf(lc)) load_bead(a, lc, X);
      else for (int i = 0; i < 6; ++i) X[i] = a.xs[(int64_t)lc * 6 + i];
      if (is_leaf(rc)) load_bead(a, rc, Y);
      else for (int i = 0; i < 6; ++i) Y[i] = a.xs[(int64_t)rc * 6 + i];
      T tr[6];
      up_node(rec, !is_leaf(lc), !is_leaf(rc), X, X + 3, Y, Y + 3, tr, tr + 3, a.out + a.roff[q]);
      for (int i = 0; i < 6; ++i) a.xs[(int64_t)q * 6 + i] = tr[i];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ downward
template <typename T>
__global__ void __launch_bounds__(kThreads) k_down_top(ApplyArgs<T> a) {
  const int32_t j = a.top_bodies[blockIdx.x];
  const int64_t nb = a.off[j] - j, ne = a.off[j + 1] - (j + 1);
  int lo, hi;
  top_range(a.top, a.counters[1], nb, ne, &lo, &hi);
  const int32_t rt = a.root[j];
  const int H = a.height[rt];
  for (int h = H; h >= 1; --h) {
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
      const int32_t q = a.top[p];
      if (a.height[q] != h) continue;
      const int32_t lc = a.cl[q], rc = a.cr[q];
      T rec[kRec];
      load_rec(a.rec + (int64_t)q * kRec, rec);
      T Lp[6];
      for (int i = 0; i < 6; ++i) Lp[i] = (q == rt) ? T(0) : a.xs[(int64_t)q * 6 + i];
      T Lx[6], Ly[6];
      down_node(rec, !is_leaf(lc), !is_leaf(rc), Lp, a.in + a.roff[q], Lx, Ly);
      if (is_leaf(lc)) store_bead(a, lc, Lx);
      else for (int i = 0; i < 6; ++i) a.xs[(int64_t)lc * 6 + i] = Lx[i];
      if (is_leaf(rc)) store_bead(a, rc, Ly);
      else for (int i = 0; i < 6; ++i) a.xs[(int64_t)rc * 6 + i] = Ly[i];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_down_tiles(ApplyArgs<T> a, int tile) {
  extern __shared__ unsigned char smem_raw[];
  T* vel = reinterpret_cast<T*>(smem_raw);
  uint16_t* list = reinterpret_cast<uint16_t*>(vel + (size_t)tile * 6);
  __shared__ int lstart[kMaxHeight + 2], lcnt[kMaxHeight + 2], hmax;
  const int ntiles = a.counters[0];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int32_t R = a.tiles[t];
    const int32_t j = body_of_node(a.off, a.m, R);
    const int64_t base = (int64_t)a.first[R] - j;
    const int nn = a.cnt[R] - 1;
    const int64_t n_body = a.off[j + 1] - a.off[j];
    if (threadIdx.x < 6)
      vel[(R - base) * 6 + threadIdx.x] =
          (a.cnt[R] < n_body) ? a.xs[(int64_t)R * 6 + threadIdx.x] : T(0);
    const int H = make_levels(a.height + base, nn, list, lstart, lcnt, &hmax);
    for (int h = H; h >= 1; --h) {
      for (int p = lstart[h] + threadIdx.x; p < lstart[h + 1]; p += blockDim.x) {
        const int li = list[p];
        const int64_t q = base + li;
        const int32_t lc = a.cl[q], rc = a.cr[q];
        T rec[kRec];
        load_rec(a.rec + q * kRec, rec);
        T Lp[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) Lp[i] = vel[(int64_t)li * 6 + i];
        T Lx[6], Ly[6];
        down_node(rec, !is_leaf(lc), !is_leaf(rc), Lp, a.in + a.roff[q], Lx, Ly);
        if (is_leaf(lc)) store_bead(a, lc, Lx);
        else {
#pragma unroll
          for (int i = 0; i < 6; ++i) vel[(lc - base) * 6 + i] = Lx[i];
        }
        if (is_leaf(rc)) store_bead(a, rc, Ly);
        else {
#pragma unroll
          for (int i = 0; i < 6; ++i) vel[(rc - base) * 6 + i] = Ly[i];
        }
      }
      __syncthreads();
    }
  }
}

template <typename T>
ApplyArgs<T> make_args(const Ctx& c, const T* rec, T* xs, const T* in, T* out) {
  ApplyArgs<T> a;
  a.off = c.off; a.m = c.m; a.N = c.N;
  a.perm = c.perm; a.cl = c.cl; a.cr = c.cr; a.cnt = c.cnt; a.first = c.first; a.roff = c.roff;
  a.height = c.height; a.tiles = c.tiles; a.top = c.top; a.counters = c.counters;
  a.top_bodies = c.top_d; a.root = c.root;
  a.rec = rec; a.xs = xs; a.in = in; a.out = out;
  return a;
}

template <typename T>
size_t tile_smem(int tile) { return (size_t)tile * (6 * sizeof(T) + sizeof(uint16_t)); }

template <typename T>
zq_status run_up(Ctx& c, const T* rec, T* xs, const T* v, T* out) {
  ApplyArgs<T> a = make_args<T>(c, rec, xs, v, out);
  const size_t smem = tile_smem<T>(c.tile);
  ZQ_CUDA_TRY(cudaFuncSetAttribute(k_up_tiles<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  time_begin(c, "up_tiles");
  k_up_tiles<T><<<c.num_sms * 4, kThreads, smem, c.stream>>>(a, c.tile);
  time_end(c, "up_tiles");
  ZQ_CUDA_TRY(cudaGetLastError());
  if (!c.top_bodies.empty()) {
    time_begin(c, "up_top");
    k_up_top<T><<<(unsigned)c.top_bodies.size(), kThreads, 0, c.stream>>>(a);
    time_end(c, "up_top");
    ZQ_CUDA_TRY(cudaGetLastError());
  }
  return ZQ_OK;
}

template <typename T>
zq_status run_down(Ctx& c, const T* rec, T* xs, const T* w, T* out) {
  ApplyArgs<T> a = make_args<T>(c, rec, xs, w, out);
  if (!c.top_bodies.empty()) {
    time_begin(c, "down_top");
    k_down_top<T><<<(unsigned)c.top_bodies.size(), kThreads, 0, c.stream>>>(a);
    time_end(c, "down_top");
    ZQ_CUDA_TRY(cudaGetLastError());
  }
  const size_t smem = tile_smem<T>(c.tile);
  ZQ_CUDA_TRY(cudaFuncSetAttribute(k_down_tiles<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  time_begin(c, "down_tiles");
  k_down_tiles<T><<<c.num_sms * 4, kThreads, smem, c.stream>>>(a, c.tile);
  time_end(c, "down_tiles");
  ZQ_CUDA_TRY(cudaGetLastError());
  return ZQ_OK;
}

}  // namespace

zq_status launch_apply_Q(Ctx& c, zq_prec prec, const void* v, int64_t /*ldv*/, void* out) {
  if (prec == ZQ_FP64)
    return run_up<double>(c, c.rec64, c.x64, static_cast<const double*>(v), static_cast<double*>(out));
  return run_up<float>(c, c.rec32, c.x32, static_cast<const float*>(v), static_cast<float*>(out));
}

zq_status launch_apply_QT(Ctx& c, zq_prec prec, const void* w, void* out, int64_t /*ldo*/) {
  if (prec == ZQ_FP64)
    return run_down<double>(c, c.rec64, c.x64, static_cast<const double*>(w), static_cast<double*>(out));
  return run_down<float>(c, c.rec32, c.x32, static_cast<const float*>(w), static_cast<float*>(out));
}

}  // namespace zq
