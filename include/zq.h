/*
 * zq.h -- C ABI of libzq: hierarchical orthogonal-complement products
 * Q~v and Q~^T w for rigid bodies on a GB300 (sm_103a).
 *
 * Method: F. Fang, J. Huang, G. Huber, J. A. McCammon, B. Zhang,
 * "Hierarchical Orthogonal Matrix Generation and Matrix-Vector
 * Multiplications in Rigid Body Simulations", arXiv 1708.08427.
 *
 * A rigid body of n beads at positions r_i has the 6 x 3n Z-matrix
 * Z = [I ... I; A_1 ... A_n], A_i f = r_i x f (Sec. 1, Eq. 1.2).  Q~ is the
 * (3n-6) x 3n matrix whose rows are an orthonormal basis of the orthogonal
 * complement of the row space of Z (Problem Statement, Sec. 1).  For m
 * bodies Q~ = diag(Q~^1, ..., Q~^m) (Sec. 1).  Q~ is never formed: a bead
 * tree (Sec. 2.1) carries one small orthogonal transform per node (Sec. 3,
 * Eq. 3.5), applied upward for Q~v (Algorithm 2, Eqs. 4.2-4.3) and
 * downward for Q~^T w (Algorithm 3, Theorem 4.3).
 *
 * Conventions shared by every call
 * --------------------------------
 * Bodies.  m bodies; body j owns beads [off[j], off[j+1]) of the bead
 *   arrays, off[0] = 0, off[m] = N, every body has at least 3 beads.
 *   N <= 700,000,000.  The offsets are a HOST array (the launch plan
 *   depends on them).
 * Coordinates.  Three DEVICE arrays x, y, z of N doubles (structure of
 *   arrays), in the caller's bead order.
 * Bead vectors (inputs of Q~, outputs of Q~^T).  Mathematically the
 *   paper's ordering f = [f_1; ...; f_N] (component 3i + a = axis a of
 *   bead i).  Physically three planes: axis a of bead i of column c sits at
 *   v[c*ldv + a*N + i], ldv >= 3N.  DEVICE memory.
 * Residue vectors (outputs of Q~, inputs of Q~^T).  R = 3N - 6m values per
 *   column: body j's residues start at sum_{i<j} (3 n_i - 6); inside a body
 *   the nodes are ordered by split position (the node whose left subtree
 *   ends at sorted bead g), and inside a node by the rows 4..k of its
 *   transform G.  Column c starts at out[c*ldo], ldo >= R.  DEVICE memory.
 * Tree.  Sec. 2.1 with the readings fixed by the oracle: the root box is
 *   each body's bounding box normalised to side 1; each coordinate is
 *   quantised to 21 bits (q = min(floor((p-lo)/(hi-lo) * 2^21), 2^21-1),
 *   q = 0 when hi == lo); bisection takes z, then y, then x at each octree
 *   level, most significant bit first; empty boxes are pruned; beads in
 *   the same 21-bit cell are separated by the bits of their body-local
 *   index; leaves are single beads.  Left child = lower half.
 * Precision.  Transforms are always built in FP64 (Eq. 3.5 LQ by
 *   Householder reflections, LAPACK dgeqrf convention; Case I by the closed
 *   form of Eqs. 3.9-3.10); an FP32 copy is kept for the FP32 applies.
 * Streams.  Every call is asynchronous on the context's stream unless noted.
 * Ownership.  The caller owns all coordinate, vector and offset buffers;
 *   the context owns the tree, the transforms and its scratch.  Apply calls
 *   never allocate.
 * Errors.  No exceptions cross the ABI.  Argument errors return at once;
 *   errors found on the device (non-finite coordinates, singular node transforms)
 *   are recorded and returned by zq_sync.
 */
#ifndef ZQ_H
#define ZQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct zq_ctx zq_ctx;

typedef enum {
  ZQ_OK = 0,
  ZQ_EINVAL = 1,        /* bad argument (NULL, sizes, n_j < 3, bad offsets) */
  ZQ_ENOMEM = 2,        /* device allocation failed */
  ZQ_ECUDA = 3,         /* a CUDA call failed; the context is unusable */
  ZQ_ESTATE = 4,        /* called out of order (apply before build) */
  ZQ_ENONFINITE = 5,    /* a coordinate is NaN or infinite (from zq_sync) */
  ZQ_WDEGENERATE = 6    /* warning: a node's T22 is singular (coincident beads,
                           or collinear beads below a node); the result is
                           orthonormal but Q~ may miss a direction */
} zq_status;

/* Arithmetic and storage of an apply.  ZQ_BF16: bfloat16 vectors with
 * FP32 arithmetic and the FP32 transforms (block form only). */
/* Arithmetic of a product.  ZQ_FP64, ZQ_FP32: the vectors and the
 * arithmetic in that type.  The block form (k right-hand sides) also takes
 * ZQ_BF16 (bfloat16 storage, FP32 arithmetic), and two tensor-core forms in
 * which each node's transform is applied to the k columns as a small
 * matrix product on the tensor cores with FP32 accumulation: ZQ_TF32 (float
 * storage, product operands rounded to TF32, a 10-bit significand) and
 * ZQ_BF16_TC (bfloat16 storage, operands in bfloat16). */
typedef enum { ZQ_FP64 = 0, ZQ_FP32 = 1, ZQ_BF16 = 2, ZQ_TF32 = 3, ZQ_BF16_TC = 4 } zq_prec;

/* Human-readable name of a status code (static storage). */
const char *zq_status_string(zq_status s);

/* Create a context on CUDA device `device` that issues all work on
 * `cuda_stream` (a cudaStream_t, NULL = legacy default stream).  The stream
 * must outlive the context. */
zq_status zq_create(zq_ctx **ctx, int device, void *cuda_stream);

/* Release all device memory of the context.  Synchronises its stream. */
zq_status zq_destroy(zq_ctx *ctx);

/* Tree of m bodies (Sec. 2.1; readings above).  off: HOST, m+1 entries.
 * x, y, z: DEVICE, N doubles each.  level_cut: the nodes of height
 * 1..level_cut are processed one height at a time across all bodies, the
 * nodes above it one thread block per body (performance only, results do
 * not depend on it; 0 = default 15; 1 <= level_cut <= 21).  Allocates the context's
 * buffers on the first call and whenever m or N grows; a later call with
 * the same sizes reuses them.  Asynchronous; bad coordinates are reported
 * by zq_sync. */
zq_status zq_build_tree_batched(zq_ctx *ctx, int64_t m, const int64_t *off, const double *x,
                                const double *y, const double *z, int32_t level_cut);

/* Single-body form: m = 1, off = {0, n}. */
zq_status zq_build_tree(zq_ctx *ctx, int64_t n, const double *x, const double *y,
                        const double *z, int32_t level_cut);

/* Node transforms in FP64 from the coordinates (Sec. 3: centroids,
 * sqrt(n_x/n), sqrt(n_y/n), the LQ of [R22 S22 sqrt(n_x n/n_y) R21] of
 * Eq. 3.5, Case I closed form Eqs. 3.9-3.10, Case II Eqs. 3.11-3.13).
 * x, y, z: DEVICE, the same bodies and bead order as the tree (the beads
 * may have moved: the tree is kept).  Writes both the FP64 and the FP32
 * copy.  Asynchronous; singular node transforms (coincident or collinear
 * beads) are reported by zq_sync. */
zq_status zq_build_transforms(zq_ctx *ctx, const double *x, const double *y, const double *z);

/* out = Q~ v for k columns (upward pass, Algorithm 2, Eqs. 4.2-4.3).
 * prec selects double (ZQ_FP64: v, out are double*) or float (ZQ_FP32:
 * float*).  v: DEVICE bead-vector planes (ldv >= 3N); out: DEVICE residue
 * vectors (ldo >= R).  Does not allocate.  ZQ_ESTATE before the first
 * zq_build_transforms. */
zq_status zq_apply_Q(zq_ctx *ctx, zq_prec prec, int64_t k, const void *v, int64_t ldv, void *out,
                     int64_t ldo);

/* out = Q~^T w for k columns (downward pass with a zero root Velocity-set,
 * Algorithm 3, Theorem 4.3, Eqs. 4.6-4.7).  w: DEVICE residue vectors
 * (ldw >= R); out: DEVICE bead-vector planes (ldo >= 3N).  Does not
 * allocate. */
zq_status zq_apply_QT(zq_ctx *ctx, zq_prec prec, int64_t k, const void *w, int64_t ldw,
                      void *out, int64_t ldo);

/* The whole orthogonal Q = [Q_Z; Q~] of every body (Sec. 3: the rows of
 * Q_Z = [I_n / sqrt(n); U] span Z's rows, Eq. 3.3; Q~ its complement).
 * zq_apply_Q_full: out = Q~ v as zq_apply_Q (one column), and
 *   root[6 j + i] = (Q_Z^j v)_i, the root Info-set [t; r] of body j (Eq. 4.4:
 *   t = sum of the body's bead vectors / sqrt(n_j), r the rotational part).
 * zq_apply_QT_full: out = Q~^T w + Q_Z^T root, the downward pass of
 *   Algorithm 3 started from the root Velocity-sets root[6 j ..] instead of
 *   zero (Theorem 4.3).
 * For every v: Q_Z^T (Q_Z v) + Q~^T (Q~ v) = v.  root: DEVICE, 6 m values of
 * the precision's type.  Does not allocate; ZQ_ESTATE before the transforms
 * of this precision exist. */
zq_status zq_apply_Q_full(zq_ctx *ctx, zq_prec prec, const void *v, void *out, void *root);
zq_status zq_apply_QT_full(zq_ctx *ctx, zq_prec prec, const void *w, const void *root, void *out);

/* The explicit Q~ (Algorithm 1, Eqs. 3.7-3.8) as a CSR matrix of R rows and
 * 3N columns.
 * Rows: the R residue rows in the order of zq_apply_Q's output (body j's
 *   rows from 3 off[j] - 6 j; inside a body node by node, each node's
 *   k - 3 rows together).
 * Columns: bead i's axis a is column 3 i + a (bead i in the caller's
 *   order, all bodies; the paper's interleaved ordering).  So Q~ times the
 *   interleaved vector [v_0; v_1; ...] equals zq_apply_Q of the planes.
 * Structure: a row of node p is nonzero only on p's n_p beads.  It holds
 *   3 n_p entries: the beads in the tree's order (ascending positions of
 *   the sorted keys, not ascending columns), three axes each.  Entries that
 *   happen to be 0 are stored.  So nnz = sum_p (k_p - 3) 3 n_p, which is
 *   O(n log n) (Sec. 3, the complexity of Algorithm 1).
 * zq_qgen_nnz: *nnz (HOST) = that count.  It needs the tree only, and
 *   synchronises the context stream.
 * zq_qgen: fills DEVICE buffers.
 *   row_ptr: R + 1 int64; row r is [row_ptr[r], row_ptr[r + 1]).
 *   col: nnz int32.
 *   val: nnz values of the precision's type.  The FP32 values are computed
 *     from the FP32 transforms in FP32.
 *   uz: optional (may be NULL), 9 N values.  Body j's U_j is the 3 x 3 n_j
 *     block of the rotational rows of Q_Z = [I / sqrt(n_j); U_j] (Eq. 3.3).
 *     It is row-major at uz[9 off[j]], column 3 i + a for local bead i.
 * Scratch of about 12 (N + nodes) bytes is allocated and freed
 * stream-ordered.  ZQ_EINVAL if 3N exceeds INT32_MAX; ZQ_ESTATE before the
 * transforms of this precision exist. */
zq_status zq_qgen_nnz(zq_ctx *ctx, int64_t *nnz);
zq_status zq_qgen(zq_ctx *ctx, zq_prec prec, int64_t *row_ptr, int32_t *col, void *val, void *uz);

/* qv = Q~ v and qtw = Q~^T w for one column each (Algorithms 2 and 3), the
 * two sweeps running concurrently (Q~^T w on a stream forked from and
 * joined back into the context stream, with its own scratch).  Layouts as
 * for zq_apply_Q / zq_apply_QT with ldv = 3N, ldw = R.  Does not allocate;
 * ZQ_ESTATE before the transforms of this precision exist. */
zq_status zq_apply_pair(zq_ctx *ctx, zq_prec prec, const void *v, void *qv, const void *w, void *qtw);

/* Products for rigidly moved bodies without rebuilding the transforms.
 * Body j moved rigidly: bead k goes to R_j r_k^j + d_j for a rotation R_j
 * and any translation d_j.  From Z's definition (Sec. 1, Eq. 1.2),
 * [R r]x = R [r]x R^T gives Z_moved blockdiag(R_j) = diag(R_j, R_j) Z_ref.
 * So Q~_ref blockdiag(R_j^T) has orthonormal rows orthogonal to the moved
 * body's Z rows: it is a valid Q~ of the moved body.  The projector
 * Q~^T Q~ is the same as after a rebuild; the basis is not.
 *   qv  = Q~_ref blockdiag(R^T) v   (each bead vector rotated by R_j^T,
 *                                     then Algorithm 2),
 *   qtw = blockdiag(R) Q~_ref^T w   (Algorithm 3, then each bead vector
 *                                     rotated by R_j).
 * Q~_ref are the transforms last built (zq_build_transforms / zq_pipeline)
 * on the reference coordinates.  R: DEVICE, 9 m doubles, body j's R_j
 * row-major at R[9 j]; it is used as given (not checked for orthogonality;
 * a non-orthogonal R_j gives rows that are not orthonormal).  Other
 * layouts as zq_apply_pair.  v/qv or w/qtw may both be NULL (not all
 * four); with both, the two sweeps run concurrently as in zq_apply_pair.
 * Does not allocate; ZQ_EINVAL for R == NULL, ZQ_ESTATE before the
 * transforms of this precision exist. */
zq_status zq_apply_rotated(zq_ctx *ctx, zq_prec prec, const double *R, const void *v, void *qv,
                           const void *w, void *qtw);

/* ------------------------------------------------------------------------
 * Block form: k right-hand sides at once (the same node transforms applied
 * to k-column blocks; Algorithms 2 and 3 column by column).
 *
 * Layout: rows of k contiguous values.  Bead vectors V[(a*N + i)*k + c]
 * (axis a of bead i, caller's bead order, column c); residue vectors
 * out[r*k + c] (r in the residue order above).  DEVICE memory.
 * prec: ZQ_FP32 (float), ZQ_BF16 (__nv_bfloat16 storage, FP32 arithmetic
 * and FP32 transforms; inputs and outputs rounded to bfloat16), ZQ_FP64
 * (double), ZQ_TF32 (float storage; per node, G (k_p x k_p, k_p <= 9) zero
 * padded to 16 x 16 times the node's k_p x k block in tiles of 8 columns by
 * warp-level mma.sync m16n8k8 with TF32 operands and FP32 accumulation),
 * ZQ_BF16_TC (bfloat16 storage; the same with m16n8k16 bfloat16 operands).
 * Each node's operands are rounded once (relative 2^-11 for TF32, 2^-8 for
 * bfloat16); the rounding errors of the heights add up through the tree
 * (orthogonal steps do not amplify them).  The transforms of the matching
 * precision must have been built (zq_build_transforms builds both; the
 * FP32 ones serve ZQ_FP32, ZQ_BF16, ZQ_TF32 and ZQ_BF16_TC), else
 * ZQ_ESTATE.
 *
 * zq_reserve_block allocates the context's block scratch for up to k_max
 * columns (6 values per node and column, 4 or 8 bytes each) and must precede
 * the block applies; they never allocate and return ZQ_ESTATE when k exceeds
 * the reservation or the tree changed size since.  1 <= k. */
zq_status zq_reserve_block(zq_ctx *ctx, zq_prec prec, int64_t k_max);
zq_status zq_apply_Q_block(zq_ctx *ctx, zq_prec prec, int64_t k, const void *V, void *out);
zq_status zq_apply_QT_block(zq_ctx *ctx, zq_prec prec, int64_t k, const void *W, void *out);

/* One step of the whole path for m bodies: the tree (Sec. 2.1), the FP64
 * node transforms (Sec. 3), then qv = Q~ v and qtw = Q~^T w (Algorithms 2
 * and 3) for one column each, in the precision `prec` (ZQ_FP32: v, qv, w,
 * qtw are float*; ZQ_FP64: double*).  Layouts as above (v, qtw: 3 planes of
 * N; qv, w: R values).  v/qv or w/qtw may both be NULL to skip that product.
 * flags:
 *   ZQ_HOST_BUFFERS  x, y, z, v, w, qv, qtw are HOST pointers (pinned for
 *                    asynchronous copies); the context stages them through
 *                    device buffers it owns (allocated on first use).
 *   ZQ_KEEP_TREE     keep the current tree (same bodies, beads moved):
 *                    only the transforms are rebuilt; m and off must match.
 *   ZQ_GRAPH         run the step as a CUDA graph: a call whose arguments
 *                    (pointers, sizes, offsets, flags, level cut) and plan
 *                    equal those of the captured step replays it with one
 *                    launch; otherwise the call captures itself (or, when
 *                    it must plan first, runs directly).  The buffers must
 *                    hold the new inputs when the replay runs, as for any
 *                    asynchronous call.  The zq_time_kernel events are
 *                    recorded in every replay.  Ignored on the legacy
 *                    default stream.
 * With both products and the vectors in the caller's order (the default
 * of zq_set_vector_order), the step moves the bead planes into the tree's
 * order around its sweeps: v is gathered through perm next to the
 * transform build (which also records the inverse permutation) and Q~^T w
 * is gathered back into the caller's order after its sweep, through two
 * 3N-value planes and N int32 indices the context owns (allocated on first
 * use and when N or the precision grows).  The results are the same
 * numbers.
 * Only the transform copy of the requested precision is refreshed, so a
 * later zq_apply_Q / zq_apply_QT must use the same precision (else
 * ZQ_ESTATE).  Asynchronous; the results are ready after zq_sync.  When m,
 * off, level_cut and prec equal the previous call's, no host
 * synchronisation or allocation happens and the call can be captured into
 * a CUDA graph (device buffers only). */
#define ZQ_HOST_BUFFERS 1
#define ZQ_KEEP_TREE 2
#define ZQ_GRAPH 4
zq_status zq_pipeline(zq_ctx *ctx, zq_prec prec, int64_t m, const int64_t *off, const double *x,
                      const double *y, const double *z, const void *v, void *qv, const void *w,
                      void *qtw, int32_t level_cut, int32_t flags);

/* Measurement hook: while set, every launch of the named kernel is
 * bracketed by records of start_event / stop_event (cudaEvent_t handles
 * owned by the caller) on the stream it is launched on.  The records are
 * external (cudaEventRecordExternal), so a captured step (ZQ_GRAPH, or a
 * caller's own capture) records them at every replay.  Names:
 * "small_tree" (the per-body tree kernels), "bead_body", "aabb", "keys",
 * "sort_radix", "sort_radix_count", "lcp", "bottom_up" (bodies over 8192
 * beads), "scan", "segments", "schedule", "build" (the whole transform
 * build), "build_level" (the Case I kernel and one launch per height up to
 * the level cut), "build_tail", "to_tree" / "from_tree" (zq_pipeline's
 * bead planes into and out of the tree's order around its sweeps),
 * "up_seg", "up_top", "down_top", "down_seg", their "_blk" block-form
 * variants, "qgen", "count_table".  When one API call launches the named
 * kernel several times, start is recorded before its first launch and
 * stop after its last launch in that call. */
zq_status zq_time_kernel(zq_ctx *ctx, const char *name, void *start_event, void *stop_event);

/* Arithmetic of the node-transform build.  ZQ_BUILD_FP64: native double
 * precision.  ZQ_BUILD_DD (default): double-single -- each value an
 * unevaluated sum of two floats (about 48 significant bits, relative
 * error ~1e-14), evaluated on the FP32 pipes with error-free
 * transformations; on this GPU FP64 runs at 1/64 of the FP32 rate.  Both
 * meet the 1e-12 parity with the FP64 CPU oracle; the FP32 and FP64
 * records the sweeps use are rounded from either.  Takes effect at the
 * next build. */
typedef enum { ZQ_BUILD_DD = 0, ZQ_BUILD_FP64 = 1 } zq_build_arith;
zq_status zq_set_build_arith(zq_ctx *ctx, zq_build_arith arith);

/* Schedule of zq_pipeline's step after the tree.  Bodies are independent
 * (Q~ is block diagonal over the bodies, Sec. 1), so the node transforms
 * (Sec. 3) and both sweeps (Algorithms 2 and 3) of one body need nothing
 * from any other body.
 *   ZQ_STEP_LEVELS (default): the transforms level by level over all bodies
 *     (one launch per height up to the level cut, then one block or warp
 *     per body), then the sweeps on segments of at most 512 beads.
 *   ZQ_STEP_FUSED: one launch; the bodies are dealt to the thread blocks
 *     largest first, each to the block with the fewest nodes so far, and a
 *     block runs its bodies' transforms with Q~ v, then Q~^T w, height by
 *     height.  Used when every
 *     body has at most 8192 beads (else the step falls back to
 *     ZQ_STEP_LEVELS).  The transform arithmetic and the node steps are the
 *     same, so both schedules give the same bits.  The records are stored
 *     in another layout: after a fused step the separate products
 *     (zq_apply_Q, ...) return ZQ_ESTATE until zq_build_transforms runs.
 * Performance only; takes effect at the next zq_pipeline call. */
typedef enum { ZQ_STEP_LEVELS = 0, ZQ_STEP_FUSED = 1 } zq_step_schedule;
zq_status zq_set_step_schedule(zq_ctx *ctx, zq_step_schedule schedule);

/* Order of the bead vectors of every product call that follows (inputs of
 * Q~, outputs of Q~^T, in every precision and form, and of zq_pipeline).
 * ZQ_ORDER_CALLER (default): bead i is the caller's bead i.  ZQ_ORDER_TREE:
 * entry s of each plane is the bead at sorted position s of the context's
 * current tree, i.e. the caller's bead perm[s] (perm from zq_get_tree);
 * the sweeps then read and write the planes without the gather through
 * perm.  The results are the same numbers, permuted.  Residue vectors are
 * not affected.  In zq_pipeline the order is that of the tree the call
 * builds (or keeps, with ZQ_KEEP_TREE); the tree is a deterministic function
 * of off and the coordinates, so a rebuild from unchanged coordinates gives
 * the same perm.  zq_qgen's columns stay in the caller's order. */
typedef enum { ZQ_ORDER_CALLER = 0, ZQ_ORDER_TREE = 1 } zq_vector_order;
zq_status zq_set_vector_order(zq_ctx *ctx, zq_vector_order order);

/* Number of kernels this context has launched since it was created (for
 * launch accounting in measurements). */
zq_status zq_launch_count(const zq_ctx *ctx, int64_t *launches);

/* Wait for the context's stream; return the first deferred device error
 * (ZQ_ENONFINITE, ZQ_WDEGENERATE) recorded since the last zq_sync, then
 * clear it. */
zq_status zq_sync(zq_ctx *ctx);

/* Sizes of the current tree: N beads, m bodies, R = 3N - 6m residues,
 * number of internal nodes N - m. */
zq_status zq_sizes(const zq_ctx *ctx, int64_t *N, int64_t *m, int64_t *R, int64_t *nodes);

/* Tree export (synchronous; HOST arrays), for checking the tree bit by bit.
 *   perm[N]            sorted position -> bead index (global).
 * Per internal node id q in [0, N - m) (body j's node with split position
 * g has id off[j] - j + g):
 *   left[q], right[q]  child codes: >= 0 internal node id, < 0 a leaf at
 *                      sorted position -1 - code;
 *   first[q]           sorted position of the node's first bead;
 *   count[q]           beads below the node;
 *   height[q]          1 + the larger child height (leaves: 0);
 *   roff[q]            residue offset (global).
 * Any pointer may be NULL to skip that array. */
zq_status zq_get_tree(zq_ctx *ctx, int32_t *perm, int32_t *left, int32_t *right, int32_t *first,
                      int32_t *count, int32_t *height, int32_t *roff);

/* Row orders of Q~ (Sec. 3).  ZQ_ROWS_INORDER: the order of every
 * product's residue vector: internal nodes by id (split position within a
 * body), each node's rows in the order of G's rows 4..k, bodies
 * concatenated.  ZQ_ROWS_PREORDER: the recursive layout of Sec. 3,
 * Q~_p = [Residue_p; diag(Q~_x, Q~_y)]: a node's rows, then those of its
 * left (x) subtree, then those of its right (y) subtree; bodies
 * concatenated.  A node has 3 rows per internal child (0, 3 or 6) in
 * either order, so a residue vector converts row block by row block:
 * y_pre[pre[q] + i] = y_in[in[q] + i]. */
typedef enum { ZQ_ROWS_INORDER = 0, ZQ_ROWS_PREORDER = 1 } zq_row_order;

/* Residue offsets of every internal node in the chosen row order, on the
 * HOST from a tree in zq_get_tree's form (no context, no device work):
 *   m bodies with bead offsets off[m + 1] (off[0] = 0, n_j >= 3);
 *   left[q], right[q] child codes of the N - m internal nodes (N = off[m]);
 *   node_off[N - m] (int64) receives the offsets;
 *   body_off[m + 1] (int64, may be NULL) the residue offset of each body,
 *   3 off[j] - 6 j, the same in both orders.
 * ZQ_EINVAL for a NULL array, m < 1, an unknown order, bad offsets, or
 * arrays that are not one binary tree per body (a child outside its body,
 * a node that is the child of two nodes, nodes not reached from the
 * body's root). */
zq_status zq_residue_offsets(int64_t m, const int64_t *off, const int32_t *left, const int32_t *right,
                             zq_row_order order, int64_t *node_off, int64_t *body_off);

/* zq_residue_offsets for the context's current tree (synchronous; HOST
 * arrays node_off[N - m], body_off[m + 1] or NULL).  ZQ_ESTATE before a
 * tree is built. */
zq_status zq_get_residue_offsets(zq_ctx *ctx, zq_row_order order, int64_t *node_off, int64_t *body_off);

/* FP64 node data export (synchronous; HOST arrays, N - m rows each, NULL
 * skips): centroid[3*q + a]; T22[6*q + i] packed lower triangle
 * (L00, L10, L11, L20, L21, L22). */
zq_status zq_get_nodes(zq_ctx *ctx, double *centroid, double *T22);

/* Node-transform export (synchronous; HOST array of (N - m) * 28 doubles):
 * per node q, rec[28*q + i]: [0] sqrt(n_x/n), [1] sqrt(n_y/n), [2..4] the
 * Householder factors tau_1..3 of Eq. 3.5's LQ (G = D H_3 H_2 H_1,
 * H_j = I - |tau_j| v_j v_j^T, v_j(j) = 1, v_j zero above j; D diagonal,
 * D_jj = -1 where the sign bit of tau_j is set (T22's diagonal made
 * nonnegative; tau_j may be -0.0), else 1), then the
 * reflector entries below the unit entry: v_1(2..k), v_2(3..k), v_3(4..k)
 * for k = 6, 9; for Case I (k = 3) entries 5..13 hold G row-major. */
zq_status zq_get_records(zq_ctx *ctx, double *rec);

/* ------------------------------------------------------------------------
 * Q~ v for one small body without allocating device memory.
 *
 * The paper has no counterpart to this entry point: it computes the same
 * product as zq_build_tree + zq_build_transforms + zq_apply_Q in FP64 for
 * ONE body, for callers that cannot allocate device
 * memory where they call it -- code inside a host framework that owns all
 * device memory through its own allocator, or a loop that runs on a fixed
 * memory budget -- and so cannot hold a zq_ctx, whose workspace grows with
 * the batch.  It needs no context: the intermediate data (tree and node
 * transforms, about 300 KB) lives in one fixed array in device memory that
 * the library declares statically, so it exists on every device the library
 * is loaded on, and the call never allocates.
 *
 *   device   CUDA device ordinal the pointers live on (0..63).
 *   stream   cudaStream_t (NULL = legacy default stream); the call is
 *            asynchronous on it.
 *   n        beads, 3 <= n <= ZQ_NOALLOC_MAX_BEADS; any other n returns
 *            ZQ_EINVAL before touching the GPU.
 *   x, y, z  DEVICE doubles [n]: bead coordinates (finite; not checked).
 *   v        DEVICE doubles [3 * n], three planes: v[a * n + i] is axis a
 *            of bead i.
 *   out      DEVICE doubles [3n - 6]: the Residues, in the order zq_apply_Q
 *            writes them for a batch holding only this body.
 * Nothing has to be zeroed by the caller: every value the kernel reads from
 * the static array is written earlier in the same call.  Coincident beads
 * are not reported (zq_sync's ZQ_WDEGENERATE has no equivalent here).
 *
 * The first call on each device looks up the address of the static array
 * (cudaGetSymbolAddress, with that device made current for the lookup, then
 * the caller's current device restored); make that first call before any
 * stream capture starts on the device.  Later calls only launch one kernel.
 * The address is kept for the life of the process: after cudaDeviceReset on
 * that device the library's module is reloaded and the kept address is no
 * longer valid, so do not call this entry point again after a reset.  The
 * kernel keeps everything per thread in registers (no local-memory stack
 * frame), so its first launch does not make the driver enlarge the
 * context's local-memory reservation.
 *
 * All calls on a device share the one array: two calls whose kernels can
 * run at the same time (different streams, or different host threads,
 * without an event or a synchronisation between them) race on it and both
 * results are undefined.  Issue the calls on one stream, or order them.
 * Returns ZQ_OK, ZQ_EINVAL (NULL pointer, n or device out of range) or
 * ZQ_ECUDA (lookup or launch failed). */
#define ZQ_NOALLOC_MAX_BEADS 2048
zq_status zq_apply_Q_noalloc(int device, void *stream, int64_t n, const double *x, const double *y,
                             const double *z, const double *v, double *out);

#ifdef __cplusplus
}
#endif

#endif /* ZQ_H */
