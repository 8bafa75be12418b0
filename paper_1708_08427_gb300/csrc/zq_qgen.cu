// zq_qgen.cu -- the explicit Q~ (Algorithm 1, Eqs. 3.7-3.8) in CSR form.
//
// Column (bead i, axis a) of Q~ is Q~ e_{3i+a}: the upward sweep of a unit
// vector.  Its Info-sets vanish off the path from bead i to the root, so
// the column is that path's walk: at every ancestor p the node transform
// (zq_node.cuh) takes the Info-set coming up from the child that holds the
// bead (the other child's is zero) to p's Info-set and p's Residue, whose
// k_p - 3 entries are column 3i + a of p's residue rows.  A residue row of
// p is nonzero only on p's beads (3 n_p entries), so Q~ has
// sum_p (k_p - 3) 3 n_p = O(n log n) nonzeros (the paper's count for
// Algorithm 1).  The root's Info-set rows 3-5 are column 3i + a of the
// rotational rows U of Q_Z = [I / sqrt(n); U] (Eq. 3.3).
//
// One thread per bead (sorted position) walks its path for the three axes
// at once; threads of one warp hold neighbouring positions, share their
// upper ancestors' records and write neighbouring entries of every row.
#include "zq_internal.cuh"
#include "zq_node.cuh"

namespace zq {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ int node_type(int32_t l, int32_t r) { return (l >= 0) + (r >= 0); }

// parent[q] for internal nodes (-1 at the roots), leaf_parent[s] for beads.
__global__ void k_parents(int64_t nodes, const int32_t* __restrict__ cl, const int32_t* __restrict__ cr,
                          int32_t* __restrict__ parent, int32_t* __restrict__ leaf_parent) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nodes) return;
  const int32_t l = cl[q], r = cr[q];
  if (l >= 0) parent[l] = (int32_t)q; else leaf_parent[leaf_pos(l)] = (int32_t)q;
  if (r >= 0) parent[r] = (int32_t)q; else leaf_parent[leaf_pos(r)] = (int32_t)q;
}

// Nonzeros of node q's residue rows: (k - 3) rows of 3 n_q entries.
__global__ void k_node_nnz(int64_t nodes, const int32_t* __restrict__ cl, const int32_t* __restrict__ cr,
                           const int32_t* __restrict__ cnt, int64_t* __restrict__ nnz) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nodes) return;
  nnz[q] = 9 * (int64_t)node_type(cl[q], cr[q]) * cnt[q];
}

// Row pointers: node q's rows (residue offset roff[q], node-id order) start
// at base[q], 3 n_q apart.
__global__ void k_row_ptr(int64_t nodes, const int32_t* __restrict__ cl, const int32_t* __restrict__ cr,
                          const int32_t* __restrict__ cnt, const int32_t* __restrict__ roff,
                          const int64_t* __restrict__ base, int64_t* __restrict__ row_ptr) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nodes) return;
  const int rows = 3 * node_type(cl[q], cr[q]);
  const int64_t len = 3 * (int64_t)cnt[q];
  for (int i = 0; i < rows; ++i) row_ptr[roff[q] + i] = base[q] + i * len;
}

struct QgenArgs {
  int64_t N;
  const int32_t* perm;
  const int32_t* bead_body;
  const int64_t* off;
  const int32_t* leaf_parent;
  const int32_t* parent;
  const int32_t* cl;
  const int32_t* cr;
  const int32_t* first;
  const int32_t* roff;
  const int32_t* pos_of;
  const uint32_t* prw;
  const int64_t* row_ptr;
  int32_t* col;
};

template <typename T, int TYPE>
__device__ __forceinline__ void path_node(const T* __restrict__ recp, bool from_x, bool xi, T (&cur)[3][6],
                                          T (&res)[3][6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T X[6], Y[6], P[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      X[e] = from_x ? cur[c][e] : T(0);
      Y[e] = from_x ? T(0) : cur[c][e];
    }
    up_node<T, TYPE>(recp, X, Y, xi, P, res[c]);
#pragma unroll
    for (int e = 0; e < 6; ++e) cur[c][e] = P[e];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_qgen(QgenArgs a, const T* __restrict__ rec, T* __restrict__ val,
                                                   T* __restrict__ uz) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.N) return;
  const int32_t bead = a.perm[s];
  T cur[3][6];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int e = 0; e < 6; ++e) cur[c][e] = T(c == e ? 1 : 0);  // leaf Info-set t = e_c
  int32_t prev = -1 - (int32_t)s;                             // the leaf's code
  int32_t p = a.leaf_parent[s];
  for (int it = 0; it < kMaxHeight && p >= 0; ++it) {
    const int32_t l = a.cl[p], r = a.cr[p];
    const int type = node_type(l, r);
    const bool from_x = l == prev;
    const T* recp = rec + 4 * (int64_t)a.prw[a.pos_of[p]];
    T res[3][6];
    if (type == 0) path_node<T, 0>(recp, from_x, false, cur, res);
    else if (type == 1) path_node<T, 1>(recp, from_x, l >= 0, cur, res);
    else path_node<T, 2>(recp, from_x, true, cur, res);
    if (type) {
      const int64_t o = 3 * (s - a.first[p]);
      const int32_t ro = a.roff[p];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (i < 3 * type) {
          const int64_t b = a.row_ptr[ro + i] + o;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            val[b + c] = res[c][i];
            a.col[b + c] = 3 * bead + c;
          }
        }
      }
    }
    prev = p;
    p = a.parent[p];
  }
  if (uz) {
    const int32_t j = a.bead_body[s];
    const int64_t o = a.off[j], n = a.off[j + 1] - o;
    T* U = uz + 9 * o;
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
      for (int c = 0; c < 3; ++c) U[e * 3 * n + 3 * (bead - o) + c] = cur[c][3 + e];
  }
}

struct Scratch {
  int32_t* parent = nullptr;
  int32_t* leaf_parent = nullptr;
  int64_t* nnz = nullptr;     // [nodes], scanned in place to the node bases
  int64_t* tmp = nullptr;     // scan workspace + the total
  int64_t tmp_words = 0;
};

zq_status alloc_scratch(Ctx& c, Scratch& S) {
  S.tmp_words = scan_tmp_words(c.nodes) + 1;
  const size_t bytes = (size_t)(c.nodes + c.N) * 4 + (size_t)(c.nodes + S.tmp_words) * 8;
  char* p = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&p), bytes, c.stream) != cudaSuccess) return ZQ_ENOMEM;
  S.nnz = reinterpret_cast<int64_t*>(p);
  S.tmp = S.nnz + c.nodes;
  S.parent = reinterpret_cast<int32_t*>(S.tmp + S.tmp_words);
  S.leaf_parent = S.parent + c.nodes;
  return ZQ_OK;
}

void free_scratch(Ctx& c, Scratch& S) {
  if (S.nnz) cudaFreeAsync(S.nnz, c.stream);
  S.nnz = nullptr;
}

// Node nonzero counts scanned to bases; the total at S.tmp[tmp_words - 1].
zq_status node_bases(Ctx& c, Scratch& S) {
  const int64_t n = c.nodes;
  k_node_nnz<<<blocks(n), kThreads, 0, c.stream>>>(n, c.cl, c.cr, c.cnt, S.nnz);
  return launch_exclusive_scan64(c, S.nnz, S.nnz, n, S.tmp, S.tmp + S.tmp_words - 1);
}

}  // namespace

zq_status launch_qgen_nnz(Ctx& c, int64_t* nnz_host) {
  Scratch S;
  ZQ_TRY_STATUS(alloc_scratch(c, S));
  zq_status st = node_bases(c, S);
  if (st == ZQ_OK && cudaMemcpyAsync(nnz_host, S.tmp + S.tmp_words - 1, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                     c.stream) != cudaSuccess)
    st = ZQ_ECUDA;
  free_scratch(c, S);
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) return ZQ_ECUDA;
  return st;
}

zq_status launch_qgen(Ctx& c, zq_prec prec, int64_t* row_ptr, int32_t* col, void* val, void* uz) {
  Scratch S;
  ZQ_TRY_STATUS(alloc_scratch(c, S));
  zq_status st = node_bases(c, S);
  const int64_t n = c.nodes;
  if (st == ZQ_OK) {
    k_row_ptr<<<blocks(n), kThreads, 0, c.stream>>>(n, c.cl, c.cr, c.cnt, c.roff, S.nnz, row_ptr);
    if (cudaMemcpyAsync(row_ptr + c.R, S.tmp + S.tmp_words - 1, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                        c.stream) != cudaSuccess)
      st = ZQ_ECUDA;
  }
  if (st == ZQ_OK) {
    if (cudaMemsetAsync(S.parent, 0xff, (size_t)n * sizeof(int32_t), c.stream) != cudaSuccess) st = ZQ_ECUDA;
  }
  if (st == ZQ_OK) {
    k_parents<<<blocks(n), kThreads, 0, c.stream>>>(n, c.cl, c.cr, S.parent, S.leaf_parent);
    QgenArgs a;
    a.N = c.N; a.perm = c.perm; a.bead_body = c.bead_body; a.off = c.off;
    a.leaf_parent = S.leaf_parent; a.parent = S.parent; a.cl = c.cl; a.cr = c.cr;
    a.first = c.first; a.roff = c.roff; a.pos_of = c.pos_of;
    a.prw = reinterpret_cast<const uint32_t*>(c.prw);
    a.row_ptr = row_ptr; a.col = col;
    time_begin(c, "qgen");
    if (prec == ZQ_FP64)
      k_qgen<double><<<blocks(c.N), kThreads, 0, c.stream>>>(a, c.rec64, static_cast<double*>(val),
                                                              static_cast<double*>(uz));
    else
      k_qgen<float><<<blocks(c.N), kThreads, 0, c.stream>>>(a, c.rec32, static_cast<float*>(val),
                                                             static_cast<float*>(uz));
    time_end(c, "qgen");
    if (cudaGetLastError() != cudaSuccess) st = ZQ_ECUDA;
  }
  free_scratch(c, S);
  return st;
}

}  // namespace zq
