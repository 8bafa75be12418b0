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
// Three threads per bead (sorted position), one per axis, walk the bead's
// path; threads of one warp hold neighbouring columns, share their upper
// ancestors' records and write neighbouring entries of every row.
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

// What the walk needs of node q, in two 16-byte words:
//   a = (record offset in 4-word units, residue offset, first position, beads)
//   b = (left child code, right child code, parent or -1, height)
struct __align__(16) NodeMeta {
  int4 a;
  int4 b;
};

__global__ void k_meta(int64_t nodes, const int32_t* __restrict__ cl, const int32_t* __restrict__ cr,
                       const int32_t* __restrict__ first, const int32_t* __restrict__ cnt,
                       const int32_t* __restrict__ roff, const uint8_t* __restrict__ height,
                       const int32_t* __restrict__ pos_of, const uint32_t* __restrict__ prw,
                       const int32_t* __restrict__ parent, NodeMeta* __restrict__ meta) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nodes) return;
  NodeMeta M;
  M.a = make_int4((int32_t)prw[pos_of[q]], roff[q], first[q], cnt[q]);
  M.b = make_int4(cl[q], cr[q], parent[q], height[q]);
  meta[q] = M;
}

struct QgenArgs {
  int64_t N;
  const int32_t* perm;
  const int32_t* bead_body;
  const int64_t* off;
  const int32_t* leaf_parent;
  const NodeMeta* meta;
  const int64_t* base;   // first entry of each node's rows
  int32_t* col;
};

// Three threads per bead, one per axis c (thread 3 t + c of the grid: the
// bead at sorted position t, column c).  Heights increase strictly along a
// path, so the walk goes height by height: at height h a thread takes its
// current ancestor if that ancestor has height h.  The lanes under one node
// take it in the same step, and lane order is the order of the node's row
// entries (3 (position - first) + c), so every row store of a warp covers
// consecutive words.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_qgen(QgenArgs a, const T* __restrict__ rec, T* __restrict__ val,
                                                   T* __restrict__ uz) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t s = g / 3;
  const int c = (int)(g - 3 * s);
  const bool live = s < a.N;
  const int32_t bead = live ? a.perm[s] : 0;
  T cur[6];
#pragma unroll
  for (int e = 0; e < 6; ++e) cur[e] = T(c == e ? 1 : 0);  // leaf Info-set t = e_c
  int32_t prev = -1 - (int32_t)s;                          // the leaf's code
  int32_t p = live ? a.leaf_parent[s] : -1;
  NodeMeta M;
  int64_t base = 0;
  if (p >= 0) {
    M = a.meta[p];
    base = a.base[p];
  }
  const int32_t colv = 3 * bead + c;
  for (int h = 1; h <= kMaxHeight; ++h) {
    if (p >= 0 && M.b.w == h) {
      const int32_t l = M.b.x, r = M.b.y;
      const int type = node_type(l, r);
      const bool from_x = l == prev;
      const T* recp = rec + 4 * (int64_t)M.a.x;
      T X[6], Y[6], P[6], res[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        X[e] = from_x ? cur[e] : T(0);
        Y[e] = from_x ? T(0) : cur[e];
      }
      if (type == 0) up_node<T, 0>(recp, X, Y, false, P, res);
      else if (type == 1) up_node<T, 1>(recp, X, Y, l >= 0, P, res);
      else up_node<T, 2>(recp, X, Y, true, P, res);
#pragma unroll
      for (int e = 0; e < 6; ++e) cur[e] = P[e];
      const int64_t len = 3 * (int64_t)M.a.w;
      const int64_t o = base + 3 * (s - M.a.z) + c;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (i < 3 * type) {
          val[o + i * len] = res[i];
          a.col[o + i * len] = colv;
        }
      }
      prev = p;
      p = M.b.z;
      if (p >= 0) {
        M = a.meta[p];
        base = a.base[p];
      }
    }
    if (!__any_sync(0xffffffffu, p >= 0)) break;
  }
  if (live && uz) {
    const int32_t j = a.bead_body[s];
    const int64_t o = a.off[j], n = a.off[j + 1] - o;
    T* U = uz + 9 * o;
#pragma unroll
    for (int e = 0; e < 3; ++e) U[e * 3 * n + 3 * (bead - o) + c] = cur[3 + e];
  }
}

struct Scratch {
  NodeMeta* meta = nullptr;   // [nodes]
  int32_t* parent = nullptr;
  int32_t* leaf_parent = nullptr;
  int64_t* nnz = nullptr;     // [nodes], scanned in place to the node bases
  int64_t* tmp = nullptr;     // scan workspace + the total
  int64_t tmp_words = 0;
};

zq_status alloc_scratch(Ctx& c, Scratch& S) {
  S.tmp_words = scan_tmp_words(c.nodes) + 1;
  const size_t bytes = (size_t)c.nodes * sizeof(NodeMeta) + (size_t)(c.nodes + S.tmp_words) * 8 +
                       (size_t)(c.nodes + c.N) * 4;
  char* p = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&p), bytes, c.stream) != cudaSuccess) return ZQ_ENOMEM;
  S.meta = reinterpret_cast<NodeMeta*>(p);
  S.nnz = reinterpret_cast<int64_t*>(S.meta + c.nodes);
  S.tmp = S.nnz + c.nodes;
  S.parent = reinterpret_cast<int32_t*>(S.tmp + S.tmp_words);
  S.leaf_parent = S.parent + c.nodes;
  return ZQ_OK;
}

void free_scratch(Ctx& c, Scratch& S) {
  if (S.meta) cudaFreeAsync(S.meta, c.stream);
  S.meta = nullptr;
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
    k_meta<<<blocks(n), kThreads, 0, c.stream>>>(n, c.cl, c.cr, c.first, c.cnt, c.roff, c.height, c.pos_of,
                                                 reinterpret_cast<const uint32_t*>(c.prw), S.parent, S.meta);
    QgenArgs a;
    a.N = c.N; a.perm = c.perm; a.bead_body = c.bead_body; a.off = c.off;
    a.leaf_parent = S.leaf_parent; a.meta = S.meta; a.base = S.nnz; a.col = col;
    time_begin(c, "qgen");
    if (prec == ZQ_FP64)
      k_qgen<double><<<blocks(3 * c.N), kThreads, 0, c.stream>>>(a, c.rec64, static_cast<double*>(val),
                                                                  static_cast<double*>(uz));
    else
      k_qgen<float><<<blocks(3 * c.N), kThreads, 0, c.stream>>>(a, c.rec32, static_cast<float*>(val),
                                                                 static_cast<float*>(uz));
    time_end(c, "qgen");
    if (cudaGetLastError() != cudaSuccess) st = ZQ_ECUDA;
  }
  free_scratch(c, S);
  return st;
}

}  // namespace zq
