/*
 * zq_oracle.c -- plain, slow FP64 CPU oracle for the hierarchical
 * orthogonal-complement products Q~v and Q~^T w of
 * Fang, Huang, Huber, McCammon and Zhang, "Hierarchical Orthogonal Matrix
 * Generation and Matrix-Vector Multiplications in Rigid Body Simulations"
 * (arXiv 1708.08427).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this code.  It shares nothing with the CUDA
 * library: no headers, no helpers, no constants.  Everything is recursive
 * and follows the paper's order of operations so it can be checked by eye.
 *
 * What it computes, per rigid body of n >= 3 beads:
 *   1. The bisection tree of Sec. 2.1 (root box = bounding box normalised to
 *      side 1, split at the midpoints, z first, then y, then x, empty boxes
 *      pruned, single beads at the leaves).
 *   2. Per internal node the transform of Sec. 3: centroid, sqrt(n_x/n),
 *      sqrt(n_y/n), the 3 x k matrix [R22 S22 sqrt(n_x n/n_y) R21] of Eq. 3.5
 *      and its LQ factorisation [T22 0] G (G k x k orthogonal); Case I
 *      (bead & bead) uses the closed form of Eqs. 3.9-3.10, Case II
 *      (body & bead) the 3 x 6 form of Eqs. 3.11-3.13.
 *   3. The upward pass of Algorithm 2 (Eqs. 4.2-4.3): Q~ v = all Residues.
 *   4. The downward pass of Algorithm 3 (Theorem 4.3, Eqs. 4.6-4.7):
 *      Q~^T w with a zero root Velocity-set.
 *   5. The explicit generation of Algorithm 1 (Eqs. 3.6-3.8, 3.10, 3.12,
 *      3.13): dense Q~ and Q_Z for small n.
 *
 * Readings of points the paper leaves open (each is also listed in the
 * design notes of the repository):
 *   - Quantisation: each coordinate is mapped to 21 bits,
 *     q = min(floor((p - lo)/(hi - lo) * 2^21), 2^21 - 1) (q = 0 when
 *     hi == lo); the bisection at depth l uses bit 20 - l/3 of the z, y, x
 *     coordinate for l % 3 = 0, 1, 2.  A bead on a midpoint goes to the
 *     upper half.  Beads that share all 63 bits are separated by the bits of
 *     their body-local index, most significant first.
 *   - Empty ghost boxes are pruned, so a bisection that leaves one side empty
 *     creates no node (single-child chains collapse).
 *   - Left child "x" = lower half, right child "y" = upper half.
 *   - Internal nodes are numbered by their split position g: the node whose
 *     left subtree ends at in-order leaf g.  Residues are stored in order of
 *     g; within a node, in the order of the rows 4..k of G.
 *   - The LQ factorisation is the Householder QR of M^T exactly as LAPACK
 *     dgeqrf/dorgqr (and hence Matlab qr) computes it, then the diagonal of R
 *     made nonnegative by flipping the signs of rows of R and of Q^T
 *     together: T22 = R(1:3,1:3)^T lower triangular with a nonnegative
 *     diagonal (the layout of Eq. 3.6), G = Q^T; a column whose part below
 *     the diagonal is exactly zero gets no reflection.  Before each
 *     reflection, a column whose entries (from the diagonal down) all have
 *     binary exponents more than 40 below that of the largest entry of M is
 *     set to 0 (rounding noise of an exact zero when M is rank-deficient;
 *     LAPACK would reflect on the noise); any other column is reduced
 *     exactly as LAPACK reduces it.
 *   - A node whose T22 comes out (numerically) singular is flagged
 *     degenerate: a diagonal entry of T22 zero or more than 33 binary
 *     orders below M's largest entry; coincident beads in Case I (d = 0)
 *     are flagged too.
 *   - Case I: G rows are the three rows of U in Eq. 3.10 with the factor
 *     [1, -1]/sqrt(2) removed: g1 = (e_x x d)/|e_x x d|, g2 = dhat x g1,
 *     g3 = -dhat, d = c_x - c_y; T22 = K G^T, which reduces to
 *     sqrt(n_x n_y/n)|d| [g2, -g1, 0].  When d has no y and z part,
 *     g1 = (e_y x d)/|e_y x d|; when d = 0, G = I and T22 = 0.
 *   - Leaves carry a 3-vector Info-set and Velocity-set (Definition 4.1,
 *     Definition 4.2 / the single-bead remark after Theorem 4.3); the
 *     transform of a node has k = 3 + 3 * (number of internal children).
 */
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define QBITS 21                 /* bits per coordinate after quantisation */
#define COORD_LEVELS (3 * QBITS) /* bisection depths driven by coordinates */
#define INDEX_BITS 32            /* bisection depths driven by the bead index */

#define LEAF(pos) (-1 - (pos))
#define IS_LEAF(code) ((code) < 0)
#define LEAF_POS(code) (-1 - (code))

typedef struct {
  int k;          /* size of G: 3 (two leaves), 6 (one leaf), 9 (none) */
  int cnt;        /* beads below the node */
  int degenerate; /* coincident beads (Case I) or singular T22 */
  double alpha;   /* sqrt(n_x / n) */
  double beta;    /* sqrt(n_y / n) */
  double c[3];    /* centroid */
  double L[9];    /* T22, 3 x 3 lower triangular, row-major */
  double G[81];   /* k x k orthogonal, row-major */
} orc_node;

typedef struct orc_body {
  int64_t n;
  double *x, *y, *z;
  int32_t *perm;   /* in-order leaf position -> body-local bead index */
  int32_t *left;   /* per internal node g: child code (>= 0 node, < 0 leaf) */
  int32_t *right;
  int32_t *first;  /* in-order leaf range of node g */
  int32_t *last;
  int32_t *height; /* leaves have height 0 */
  int64_t *roff;   /* residue offset of node g */
  int32_t root;
  orc_node *node;
} orc_body;

/* ------------------------------------------------------------------ */
/* 1. Tree (Sec. 2.1)                                                  */
/* ------------------------------------------------------------------ */

/* q[3*i + a] for axis a = 0 (x), 1 (y), 2 (z): the root box normalised to
 * side 1 in each direction (Sec. 2.1), then 21-bit fixed point. */
static void quantise(const orc_body *b, uint32_t *q) {
  const double *p[3] = {b->x, b->y, b->z};
  for (int a = 0; a < 3; ++a) {
    double lo = p[a][0], hi = p[a][0];
    for (int64_t i = 1; i < b->n; ++i) {
      if (p[a][i] < lo) lo = p[a][i];
      if (p[a][i] > hi) hi = p[a][i];
    }
    for (int64_t i = 0; i < b->n; ++i) {
      uint32_t v = 0;
      if (hi > lo) {
        double t = (p[a][i] - lo) / (hi - lo);
        double s = floor(t * (double)(1u << QBITS));
        v = (s >= (double)((1u << QBITS) - 1)) ? ((1u << QBITS) - 1) : (uint32_t)s;
      }
      q[3 * i + a] = v;
    }
  }
}

/* Which half bead i falls in at bisection depth l: 0 = lower, 1 = upper.
 * Depths 0, 1, 2 split z, y, x of the first octree level (the "ghost"
 * nodes of the Comment in Sec. 2.1), depths 3, 4, 5 the next level, ... */
static int half(const uint32_t *q, int32_t i, int l) {
  if (l < COORD_LEVELS) {
    int bit = QBITS - 1 - l / 3;
    int axis = 2 - l % 3; /* z, then y, then x */
    return (int)((q[3 * i + axis] >> bit) & 1u);
  }
  int bit = INDEX_BITS - 1 - (l - COORD_LEVELS);
  return (int)(((uint32_t)i >> bit) & 1u);
}

/* Recursive bisection of the bead set S (cnt beads) starting at depth l;
 * its leaves take in-order positions pos, pos+1, ...  Returns the code of
 * the subtree root. */
static int32_t bisect(orc_body *b, const uint32_t *q, int32_t *S, int32_t cnt,
                      int l, int32_t pos, int32_t *tmp) {
  if (cnt == 1) {
    b->perm[pos] = S[0];
    return LEAF(pos);
  }
  int32_t n0 = 0;
  for (; l < COORD_LEVELS + INDEX_BITS; ++l) {
    n0 = 0;
    for (int32_t i = 0; i < cnt; ++i) n0 += (half(q, S[i], l) == 0);
    if (n0 > 0 && n0 < cnt) break; /* an empty side is pruned */
  }
  if (l == COORD_LEVELS + INDEX_BITS) abort(); /* duplicate bead index */
  int32_t a = 0, c = n0;
  for (int32_t i = 0; i < cnt; ++i) {
    if (half(q, S[i], l) == 0) tmp[a++] = S[i];
    else tmp[c++] = S[i];
  }
  memcpy(S, tmp, sizeof(int32_t) * (size_t)cnt);
  int32_t lc = bisect(b, q, S, n0, l + 1, pos, tmp);
  int32_t rc = bisect(b, q, S + n0, cnt - n0, l + 1, pos + n0, tmp);
  int32_t g = pos + n0 - 1;
  b->left[g] = lc;
  b->right[g] = rc;
  b->first[g] = pos;
  b->last[g] = pos + cnt - 1;
  int32_t hl = IS_LEAF(lc) ? 0 : b->height[lc];
  int32_t hr = IS_LEAF(rc) ? 0 : b->height[rc];
  b->height[g] = 1 + (hl > hr ? hl : hr);
  return g;
}

/* ------------------------------------------------------------------ */
/* 2. Node transforms (Sec. 3)                                         */
/* ------------------------------------------------------------------ */

/* Householder LQ of the 3 x k matrix M (row-major): M = [L 0] G with L
 * lower triangular and G k x k orthogonal.  Computed as the QR
 * factorisation M^T = Q R of LAPACK dgeqrf (dlarfg reflectors) with
 * L = R(1:3,1:3)^T and G = Q^T (Eq. 3.5). */
static void lq(const double *M, int k, double *L, double *G) {
  double A[9][3];
  double v[3][9];
  double tau[3];
  int emax = INT_MIN;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < 3; ++j) {
      A[i][j] = M[j * k + i];
      if (A[i][j] != 0.0 && ilogb(A[i][j]) > emax) emax = ilogb(A[i][j]);
    }
  /* Numerical rank decision: when every entry of the column to be
   * reduced (rows j..k-1) has a binary exponent more than 40 below that of
   * the largest entry of M, the column is rounding noise of an exact zero
   * (rank-deficient M: collinear or coincident beads below the node) and
   * is set to zero, so that the factorisation is a deterministic function
   * of the geometry.  A column with any entry above that level is reduced
   * exactly as LAPACK does, small entries included. */
  for (int j = 0; j < 3; ++j) {
    int noise = 1;
    for (int i = j; i < k; ++i)
      if (A[i][j] != 0.0 && ilogb(A[i][j]) >= emax - 40) noise = 0;
    if (noise)
      for (int i = j; i < k; ++i) A[i][j] = 0.0;
    for (int i = 0; i < k; ++i) v[j][i] = 0.0;
    v[j][j] = 1.0;
    double xn2 = 0.0;
    for (int i = j + 1; i < k; ++i) xn2 += A[i][j] * A[i][j];
    if (xn2 == 0.0) { /* nothing below the diagonal: H_j = I */
      tau[j] = 0.0;
      continue;
    }
    double alpha = A[j][j];
    double norm = sqrt(alpha * alpha + xn2);
    double beta = (alpha >= 0.0) ? -norm : norm;
    tau[j] = (beta - alpha) / beta;
    for (int i = j + 1; i < k; ++i) v[j][i] = A[i][j] / (alpha - beta);
    A[j][j] = beta;
    for (int i = j + 1; i < k; ++i) A[i][j] = 0.0;
    for (int c = j + 1; c < 3; ++c) { /* A <- H_j A on the other columns */
      double w = 0.0;
      for (int i = j; i < k; ++i) w += v[j][i] * A[i][c];
      for (int i = j; i < k; ++i) A[i][c] -= tau[j] * w * v[j][i];
    }
  }
  /* Nonnegative diagonal of R: row j of R and column j of Q (row j of G)
   * change sign together, which leaves M = [T22 0] G unchanged. */
  int flip[3];
  for (int j = 0; j < 3; ++j) {
    flip[j] = A[j][j] < 0.0;
    if (flip[j])
      for (int c = j; c < 3; ++c) A[j][c] = -A[j][c];
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) L[3 * r + c] = (c <= r) ? A[c][r] : 0.0;
  /* G = Q^T = H_3 H_2 H_1 (each H_j symmetric): apply H_1, H_2, H_3 to I. */
  for (int r = 0; r < k; ++r)
    for (int c = 0; c < k; ++c) G[r * k + c] = (r == c) ? 1.0 : 0.0;
  for (int j = 0; j < 3; ++j) {
    for (int c = 0; c < k; ++c) {
      double w = 0.0;
      for (int i = 0; i < k; ++i) w += v[j][i] * G[i * k + c];
      for (int i = 0; i < k; ++i) G[i * k + c] -= tau[j] * w * v[j][i];
    }
  }
  for (int j = 0; j < 3; ++j)
    if (flip[j])
      for (int c = 0; c < k; ++c) G[j * k + c] = -G[j * k + c];
}

/* Rank test of Eq. 3.5's M after its factorisation (no pivoting, so a
 * rank loss can show at any pivot): the node is flagged when a diagonal
 * entry of T22 is zero or its binary exponent is more than 33 below that of
 * M's largest entry (below about 1e-10 of max |M|): collinear or coincident
 * beads below the node. */
static int rank_deficient(const double *M, int k, const double *L) {
  int emax = INT_MIN;
  for (int i = 0; i < 3 * k; ++i)
    if (M[i] != 0.0 && ilogb(M[i]) > emax) emax = ilogb(M[i]);
  for (int j = 0; j < 3; ++j)
    if (L[4 * j] == 0.0 || ilogb(L[4 * j]) < emax - 33) return 1;
  return 0;
}

/* Case I, bead & bead (Eqs. 3.9-3.10).  d = c_x - c_y, sk = sqrt(n_x n_y/n). */
static void case_one(const double d[3], double sk, double *L, double *G, int *degenerate) {
  double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  memset(L, 0, 9 * sizeof(double));
  if (dn == 0.0) {
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) G[3 * r + c] = (r == c) ? 1.0 : 0.0;
    *degenerate = 1;
    return;
  }
  double h[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
  double g1[3];
  if (d[1] != 0.0 || d[2] != 0.0) { /* e_x x d, first row of U in Eq. 3.10 */
    double s = sqrt(d[1] * d[1] + d[2] * d[2]);
    g1[0] = 0.0;
    g1[1] = -d[2] / s;
    g1[2] = d[1] / s;
  } else { /* d along x: e_y x d */
    double s = fabs(d[0]);
    g1[0] = 0.0;
    g1[1] = 0.0;
    g1[2] = -d[0] / s;
  }
  double g2[3] = {h[1] * g1[2] - h[2] * g1[1], h[2] * g1[0] - h[0] * g1[2],
                  h[0] * g1[1] - h[1] * g1[0]};
  for (int a = 0; a < 3; ++a) {
    G[0 + a] = g1[a];
    G[3 + a] = g2[a];
    G[6 + a] = -h[a];
  }
  /* T22 = K G^T with K = sk [d]x: K g1 = sk |d| g2, K g2 = -sk |d| g1,
   * K g3 = 0 (rank two, as noted after Eq. 3.10). */
  double s = sk * dn;
  for (int a = 0; a < 3; ++a) {
    L[3 * a + 0] = s * g2[a];
    L[3 * a + 1] = -s * g1[a];
    L[3 * a + 2] = 0.0;
  }
}

static void child_info(const orc_body *b, int32_t code, int *cnt, const double **c,
                       double cb[3], const double **L) {
  if (IS_LEAF(code)) {
    int32_t i = b->perm[LEAF_POS(code)];
    cb[0] = b->x[i];
    cb[1] = b->y[i];
    cb[2] = b->z[i];
    *cnt = 1;
    *c = cb;
    *L = NULL;
  } else {
    const orc_node *nd = &b->node[code];
    *cnt = nd->cnt;
    *c = nd->c;
    *L = nd->L;
  }
}

/* Post-order: the transform of node g needs those of its children
 * (Algorithm 1 / Algorithm 2 recurse first). */
static void transform(orc_body *b, int32_t code) {
  if (IS_LEAF(code)) return;
  int32_t g = code;
  transform(b, b->left[g]);
  transform(b, b->right[g]);
  orc_node *p = &b->node[g];
  int nx, ny;
  const double *cx, *cy, *Lx, *Ly;
  double bx[3], by[3];
  child_info(b, b->left[g], &nx, &cx, bx, &Lx);
  child_info(b, b->right[g], &ny, &cy, by, &Ly);
  int n = nx + ny;
  p->cnt = n;
  p->degenerate = 0;
  for (int a = 0; a < 3; ++a) p->c[a] = ((double)nx * cx[a] + (double)ny * cy[a]) / (double)n;
  p->alpha = sqrt((double)nx / (double)n);
  p->beta = sqrt((double)ny / (double)n);
  /* sqrt(n_x n / n_y) R21 with R21 = [c_x - c_p]x and
   * c_x - c_p = (n_y / n)(c_x - c_y) equals sqrt(n_x n_y / n) [c_x - c_y]x. */
  double d[3] = {cx[0] - cy[0], cx[1] - cy[1], cx[2] - cy[2]};
  double sk = sqrt((double)nx * (double)ny / (double)n);
  if (Lx == NULL && Ly == NULL) {
    p->k = 3;
    case_one(d, sk, p->L, p->G, &p->degenerate);
    return;
  }
  int k = 3 + (Lx ? 3 : 0) + (Ly ? 3 : 0);
  double M[27];
  int col = 0;
  if (Lx)
    for (int c = 0; c < 3; ++c, ++col)
      for (int r = 0; r < 3; ++r) M[r * k + col] = Lx[3 * r + c];
  if (Ly)
    for (int c = 0; c < 3; ++c, ++col)
      for (int r = 0; r < 3; ++r) M[r * k + col] = Ly[3 * r + c];
  /* K = sk [d]x, [d]x = [[0, -d_z, d_y], [d_z, 0, -d_x], [-d_y, d_x, 0]] */
  double K[9] = {0.0, -d[2], d[1], d[2], 0.0, -d[0], -d[1], d[0], 0.0};
  for (int c = 0; c < 3; ++c, ++col)
    for (int r = 0; r < 3; ++r) M[r * k + col] = sk * K[3 * r + c];
  p->k = k;
  lq(M, k, p->L, p->G);
  p->degenerate = rank_deficient(M, k, p->L);
}

/* ------------------------------------------------------------------ */
/* Construction / queries                                              */
/* ------------------------------------------------------------------ */

void orc_body_free(orc_body *b) {
  if (!b) return;
  free(b->x); free(b->y); free(b->z);
  free(b->perm); free(b->left); free(b->right); free(b->first); free(b->last);
  free(b->height); free(b->roff); free(b->node);
  free(b);
}

/* Build the tree and all node transforms of one body.  Returns NULL for
 * n < 3 or on allocation failure. */
orc_body *orc_body_new(int64_t n, const double *x, const double *y, const double *z) {
  if (n < 3 || n > INT32_MAX) return NULL;
  orc_body *b = (orc_body *)calloc(1, sizeof(orc_body));
  if (!b) return NULL;
  b->n = n;
  size_t nn = (size_t)n;
  b->x = malloc(nn * sizeof(double));
  b->y = malloc(nn * sizeof(double));
  b->z = malloc(nn * sizeof(double));
  b->perm = malloc(nn * sizeof(int32_t));
  b->left = malloc(nn * sizeof(int32_t));
  b->right = malloc(nn * sizeof(int32_t));
  b->first = malloc(nn * sizeof(int32_t));
  b->last = malloc(nn * sizeof(int32_t));
  b->height = malloc(nn * sizeof(int32_t));
  b->roff = malloc(nn * sizeof(int64_t));
  b->node = calloc(nn, sizeof(orc_node));
  uint32_t *q = malloc(3 * nn * sizeof(uint32_t));
  int32_t *S = malloc(nn * sizeof(int32_t));
  int32_t *tmp = malloc(nn * sizeof(int32_t));
  if (!b->x || !b->y || !b->z || !b->perm || !b->left || !b->right || !b->first ||
      !b->last || !b->height || !b->roff || !b->node || !q || !S || !tmp) {
    free(q); free(S); free(tmp);
    orc_body_free(b);
    return NULL;
  }
  memcpy(b->x, x, nn * sizeof(double));
  memcpy(b->y, y, nn * sizeof(double));
  memcpy(b->z, z, nn * sizeof(double));
  quantise(b, q);
  for (int64_t i = 0; i < n; ++i) S[i] = (int32_t)i;
  b->root = bisect(b, q, S, (int32_t)n, 0, 0, tmp);
  free(q); free(S); free(tmp);
  /* Residue sizes 0 / 3 / 6 (Case I / Case II / general), stored in order
   * of the split position. */
  int64_t off = 0;
  for (int64_t g = 0; g < n - 1; ++g) {
    b->roff[g] = off;
    off += 3 * (!IS_LEAF(b->left[g]) + !IS_LEAF(b->right[g]));
  }
  if (off != 3 * n - 6) abort();
  transform(b, b->root);
  return b;
}

int64_t orc_body_n(const orc_body *b) { return b->n; }

void orc_body_tree(const orc_body *b, int32_t *perm, int32_t *left, int32_t *right,
                   int32_t *first, int32_t *last, int32_t *height, int64_t *roff,
                   int32_t *root) {
  size_t n = (size_t)b->n;
  memcpy(perm, b->perm, n * sizeof(int32_t));
  memcpy(left, b->left, (n - 1) * sizeof(int32_t));
  memcpy(right, b->right, (n - 1) * sizeof(int32_t));
  memcpy(first, b->first, (n - 1) * sizeof(int32_t));
  memcpy(last, b->last, (n - 1) * sizeof(int32_t));
  memcpy(height, b->height, (n - 1) * sizeof(int32_t));
  memcpy(roff, b->roff, (n - 1) * sizeof(int64_t));
  *root = b->root;
}

/* Node g: k, count, degenerate flag, alpha/beta, centroid, T22, G (k*k). */
void orc_body_node(const orc_body *b, int64_t g, int32_t *k, int32_t *cnt, int32_t *degenerate,
                   double *alpha_beta, double *c, double *L, double *G) {
  const orc_node *p = &b->node[g];
  *k = p->k;
  *cnt = p->cnt;
  *degenerate = p->degenerate;
  alpha_beta[0] = p->alpha;
  alpha_beta[1] = p->beta;
  memcpy(c, p->c, 3 * sizeof(double));
  memcpy(L, p->L, 9 * sizeof(double));
  memcpy(G, p->G, (size_t)(p->k * p->k) * sizeof(double));
}

/* T22 (row-major 3 x 3) and centroid of every node, by split position:
 * the tests take the conditioning of each node's factorisation from them. */
void orc_body_nodes_all(const orc_body *b, double *L, double *c) {
  for (int64_t g = 0; g < b->n - 1; ++g) {
    memcpy(L + 9 * g, b->node[g].L, 9 * sizeof(double));
    memcpy(c + 3 * g, b->node[g].c, 3 * sizeof(double));
  }
}

/* Node-level entry points, used by the tests to pin single steps. */
void orc_lq(const double *M, int32_t k, double *L, double *G) { lq(M, k, L, G); }

void orc_case_one(const double *d, double sk, double *L, double *G, int32_t *degenerate) {
  int dg = 0;
  case_one(d, sk, L, G, &dg);
  *degenerate = dg;
}

/* ------------------------------------------------------------------ */
/* 3. Upward pass: Q~ v (Algorithm 2, Eqs. 4.2-4.3)                    */
/* ------------------------------------------------------------------ */

/* Vectors use the paper's ordering f = [f_1; ...; f_n]: component 3i + a
 * is axis a of bead i.  info = [t; r]: t the translational part
 * I_{n_p} f, r = U f (absent for a leaf). */
static void upward(const orc_body *b, int32_t code, const double *f, double *res,
                   double t[3], double r[3]) {
  if (IS_LEAF(code)) {
    int32_t i = b->perm[LEAF_POS(code)];
    for (int a = 0; a < 3; ++a) t[a] = f[3 * (int64_t)i + a];
    return;
  }
  int32_t g = code;
  double tx[3], rx[3], ty[3], ry[3];
  upward(b, b->left[g], f, res, tx, rx);
  upward(b, b->right[g], f, res, ty, ry);
  const orc_node *p = &b->node[g];
  double u[9];
  int k = 0;
  if (!IS_LEAF(b->left[g]))
    for (int a = 0; a < 3; ++a) u[k++] = rx[a];
  if (!IS_LEAF(b->right[g]))
    for (int a = 0; a < 3; ++a) u[k++] = ry[a];
  for (int a = 0; a < 3; ++a) {
    t[a] = p->alpha * tx[a] + p->beta * ty[a];
    u[k++] = p->beta * tx[a] - p->alpha * ty[a];
  }
  double y[9];
  for (int i = 0; i < k; ++i) {
    y[i] = 0.0;
    for (int j = 0; j < k; ++j) y[i] += p->G[i * k + j] * u[j];
  }
  for (int a = 0; a < 3; ++a) r[a] = y[a];
  for (int i = 3; i < k; ++i) res[b->roff[g] + (i - 3)] = y[i];
}

/* out = Q~ f (3n - 6 values); root6 (may be NULL) receives the root
 * Info-set Q_Z f = [t; r]. */
void orc_body_apply_Q(const orc_body *b, const double *f, double *out, double *root6) {
  double t[3], r[3];
  upward(b, b->root, f, out, t, r);
  if (root6) {
    for (int a = 0; a < 3; ++a) {
      root6[a] = t[a];
      root6[3 + a] = r[a];
    }
  }
}

/* ------------------------------------------------------------------ */
/* 4. Downward pass: Q~^T w (Algorithm 3, Theorem 4.3)                 */
/* ------------------------------------------------------------------ */

static void downward(const orc_body *b, int32_t code, const double Lp[6], const double *w,
                     double *out) {
  if (IS_LEAF(code)) { /* a single bead: its velocity is L_p */
    int32_t i = b->perm[LEAF_POS(code)];
    for (int a = 0; a < 3; ++a) out[3 * (int64_t)i + a] = Lp[a];
    return;
  }
  int32_t g = code;
  const orc_node *p = &b->node[g];
  int k = p->k;
  double z[9], y[9];
  for (int a = 0; a < 3; ++a) z[a] = Lp[3 + a];
  for (int i = 3; i < k; ++i) z[i] = w[b->roff[g] + (i - 3)];
  for (int i = 0; i < k; ++i) { /* y = G^T z */
    y[i] = 0.0;
    for (int j = 0; j < k; ++j) y[i] += p->G[j * k + i] * z[j];
  }
  double Lx[6] = {0}, Ly[6] = {0};
  int idx = 0;
  if (!IS_LEAF(b->left[g]))
    for (int a = 0; a < 3; ++a) Lx[3 + a] = y[idx++];
  if (!IS_LEAF(b->right[g]))
    for (int a = 0; a < 3; ++a) Ly[3 + a] = y[idx++];
  for (int a = 0; a < 3; ++a) {
    double sigma = y[idx + a];
    Lx[a] = p->alpha * Lp[a] + p->beta * sigma;
    Ly[a] = p->beta * Lp[a] - p->alpha * sigma;
  }
  downward(b, b->left[g], Lx, w, out);
  downward(b, b->right[g], Ly, w, out);
}

/* out = Q~^T w + Q_Z^T root6 (3n values).  root6 = NULL means a zero root
 * Velocity-set, i.e. out = Q~^T w. */
void orc_body_apply_QT(const orc_body *b, const double *w, const double *root6, double *out) {
  double L0[6] = {0, 0, 0, 0, 0, 0};
  if (root6)
    for (int a = 0; a < 6; ++a) L0[a] = root6[a];
  downward(b, b->root, L0, w, out);
}

/* ------------------------------------------------------------------ */
/* 5. Explicit generation (Algorithm 1)                                */
/* ------------------------------------------------------------------ */

/* Returns U of node `code` as a 3 x 3cnt matrix over the node's beads in
 * in-order position (column 3*(pos - first) + a); writes the node's
 * Residue rows into Qt ((3n-6) x 3n, columns in bead order). */
static double *qgen(const orc_body *b, int32_t code, double *Qt) {
  if (IS_LEAF(code)) return NULL; /* a leaf has U = 0 (Algorithm 1) */
  int32_t g = code;
  const orc_node *p = &b->node[g];
  int32_t lc = b->left[g], rc = b->right[g];
  double *Ux = qgen(b, lc, Qt);
  double *Uy = qgen(b, rc, Qt);
  int nx = IS_LEAF(lc) ? 1 : b->node[lc].cnt;
  int ny = IS_LEAF(rc) ? 1 : b->node[rc].cnt;
  int n = nx + ny, k = p->k;
  int64_t cols = 3 * (int64_t)n;
  /* C' = [V 0; 0 W; sqrt(n_y/n) I_{n_x}, -sqrt(n_x/n) I_{n_y}] (Theorem 3.2),
   * with the V / W block dropped for a leaf child (Case II, Case I). */
  double *C = calloc((size_t)k * (size_t)cols, sizeof(double));
  int row = 0;
  if (Ux) {
    for (int a = 0; a < 3; ++a)
      for (int64_t c = 0; c < 3 * (int64_t)nx; ++c) C[(row + a) * cols + c] = Ux[a * 3 * nx + c];
    row += 3;
  }
  if (Uy) {
    for (int a = 0; a < 3; ++a)
      for (int64_t c = 0; c < 3 * (int64_t)ny; ++c)
        C[(row + a) * cols + 3 * nx + c] = Uy[a * 3 * ny + c];
    row += 3;
  }
  for (int a = 0; a < 3; ++a) {
    for (int i = 0; i < nx; ++i) C[(row + a) * cols + 3 * i + a] = p->beta / sqrt((double)nx);
    for (int i = 0; i < ny; ++i) C[(row + a) * cols + 3 * (nx + i) + a] = -p->alpha / sqrt((double)ny);
  }
  free(Ux);
  free(Uy);
  /* [U; Residue] = G C' (Eqs. 3.7-3.8, 3.10, 3.12-3.13) */
  double *U = calloc(3 * (size_t)cols, sizeof(double));
  int64_t n3 = 3 * b->n;
  for (int i = 0; i < k; ++i) {
    for (int64_t c = 0; c < cols; ++c) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += p->G[i * k + j] * C[j * cols + c];
      if (i < 3) {
        U[i * cols + c] = s;
      } else {
        int64_t pos = b->first[g] + c / 3;
        int64_t bead = b->perm[pos];
        Qt[(b->roff[g] + i - 3) * n3 + 3 * bead + c % 3] = s;
      }
    }
  }
  free(C);
  return U;
}

/* Dense Q~ ((3n-6) x 3n) and Q_Z (6 x 3n) of one body, row-major, columns in
 * the paper's bead ordering. */
void orc_body_qgen(const orc_body *b, double *Qt, double *QZ) {
  int64_t n = b->n, n3 = 3 * n;
  memset(Qt, 0, (size_t)(n3 - 6) * (size_t)n3 * sizeof(double));
  double *U = qgen(b, b->root, Qt);
  memset(QZ, 0, 6 * (size_t)n3 * sizeof(double));
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) QZ[a * n3 + 3 * i + a] = 1.0 / sqrt((double)n);
  for (int a = 0; a < 3; ++a)
    for (int64_t c = 0; c < n3; ++c) {
      int64_t pos = c / 3;
      int64_t bead = b->perm[pos];
      QZ[(3 + a) * n3 + 3 * bead + c % 3] = U[a * n3 + c];
    }
  free(U);
}

/* ------------------------------------------------------------------ */
/* Many bodies: Q~ = diag(Q~^1, ..., Q~^m) (Sec. 1)                    */
/* ------------------------------------------------------------------ */

/* Bodies are given by offsets off[0..m] into the bead arrays.  Vectors:
 * f and the Q~^T result use the paper's interleaved ordering over all
 * beads; residues of body j start at sum_{i<j} (3 n_i - 6).  Returns 0, or
 * -1 if a body has fewer than 3 beads or memory runs out. */
int orc_batch_apply(int64_t m, const int64_t *off, const double *x, const double *y,
                    const double *z, const double *f, double *qf, const double *w,
                    double *qtw) {
  int64_t roff = 0;
  for (int64_t j = 0; j < m; ++j) {
    int64_t o = off[j], n = off[j + 1] - off[j];
    orc_body *b = orc_body_new(n, x + o, y + o, z + o);
    if (!b) return -1;
    if (f && qf) orc_body_apply_Q(b, f + 3 * o, qf + roff, NULL);
    if (w && qtw) orc_body_apply_QT(b, w + roff, NULL, qtw + 3 * o);
    roff += 3 * n - 6;
    orc_body_free(b);
  }
  return 0;
}
