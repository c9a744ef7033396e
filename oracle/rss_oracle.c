/*
 * rss_oracle.c -- plain, slow FP64 CPU oracle for the strong recursive
 * skeletonization factorization (RS-S) of Minden, Ho, Damle & Ying,
 * "A recursive skeletonization factorization based on strong admissibility".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; it is used by the tests, by the package smoke check and
 * by the benchmark's CPU baseline.  It shares no code with the CUDA path.
 *
 * Design: the oracle keeps the *whole* current matrix A (N x N, FP64,
 * row-major) and performs every strong skeletonization step Z(A;B) on it
 * exactly as Sec. 3.1 writes it (ID of the stacked far-field block, the row
 * operation U_T, the column operation L_T, then block elimination of the
 * redundant DOFs, Sec. 2.1).  Because the whole matrix is kept, Theorem 3.1
 * and Corollary 3.2 can be checked as invariants instead of being relied on.
 * Memory is O(N^2): use it for N up to ~16k.
 *
 * Readings of points where the paper is silent (each also listed in the
 * project's design notes):
 *   - matrix: A = diag*I + w*K with K_ii := 0 (second-kind form);
 *   - tree: root [0,1]^d, split a node while it holds more than leaf_size
 *     points (max depth 20); integer cell of x at depth t is
 *     floor(x * 2^t) clamped to [0, 2^t - 1]; child index = sum_d bit_d << d;
 *     DOF (tree) order = stable partition, pre-order, children ascending;
 *   - levels: depths t = maxdepth .. 2 (Algorithm 1 runs l = 1 .. L-2);
 *     a box at depth t is a tree node of depth t;
 *   - each active DOF is classified against a box by the Chebyshev distance
 *     of its own depth-t cell: 0 in B, 1 near (N), 2 the ring inside the
 *     proxy surface (O), >= 3 outside it (P) (Fig. 2, Sec. 3.2);
 *   - box order within a level: colour-major with 3^d colours
 *     c = sum_d (coord_d mod 3) 3^d, Morton order within a colour;
 *   - proxy surface: circle/sphere of radius 2.5 box sides about the box
 *     centre (Sec. 3.2); 2D: n_p equispaced angles; 3D: Fibonacci sphere;
 *     proxy rows scaled by w like the matrix entries;
 *   - ID matrix: [A_OB; A_BO^T; w K(Gamma,B); w K(B,Gamma)^T] (Eq. 3.1 with
 *     the proxy replacement of Eq. 3.6, both halves kept);
 *   - hybrid (RS-WS, Sec. 3.4, Algorithm 2): a weak step compresses the
 *     box's interactions with its whole complement, [A_XB; A_BX^T; proxy
 *     rows] with X = N u O (the cells inside the proxy surface), drops every
 *     coupling of R outside the box and eliminates R against J = S; each
 *     depth runs a weak pass over its boxes, then the strong pass; a last
 *     weak pass runs at depth 1 (the paper's practice);
 *   - ID by Householder QR with greedy column pivoting, pivot = largest
 *     trailing column norm, recomputed every step, ties to the lowest
 *     column; rank k = #{j : |R_jj| > eps |R_11|}; T = R11^{-1} R12;
 *   - X_RR is factored by LU with partial pivoting (Sec. 2.1 recommends a
 *     factorization over the inverse); the top block likewise.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Kernel and matrix entries (Sec. 1, Eq. 1.3; Sec. 4 Examples 1-2)           */
/* ------------------------------------------------------------------------ */

/* K(x - y): kind 0: -log|z|/(2 pi) (2D Laplace), kind 1: 1/(4 pi |z|). */
static double kfun(int kind, int dim, const double *x, const double *y) {
  double r2 = 0.0;
  for (int d = 0; d < dim; d++) {
    double z = x[d] - y[d];
    r2 += z * z;
  }
  double r = sqrt(r2);
  if (kind == 0) return -log(r) / (2.0 * ORC_PI);
  return 1.0 / (4.0 * ORC_PI * r);
}

typedef struct {
  int kind, dim;
  double diag, w;
} okern;

/* Entry A_ij = diag (i == j) or w K(x_i - x_j). */
static double entry(const okern *kn, const double *x, int64_t i, int64_t j) {
  if (i == j) return kn->diag;
  return kn->w * kfun(kn->kind, kn->dim, x + i * kn->dim, x + j * kn->dim);
}

/* ------------------------------------------------------------------------ */
/* Tree (Sec. 3, Sec. 4: adaptive quad/octree refined to n_occ per leaf)     */
/* ------------------------------------------------------------------------ */

typedef struct {
  int dim, leaf;
  int64_t n;
  int64_t *perm;  /* perm[g] = original index of tree-order DOF g */
  double *x;      /* tree-ordered points, n*dim */
  int nnode, cap;
  int *depth, *parent, *coord; /* coord: 3 per node */
  int64_t *start, *count;
  int maxdepth;
} otree;

static int64_t cellc(double v, int t) {
  int64_t m = (int64_t)1 << t;
  int64_t c = (int64_t)floor(v * (double)m);
  if (c < 0) c = 0;
  if (c > m - 1) c = m - 1;
  return c;
}

static int new_node(otree *T, int depth, int parent, const int *coord, int64_t start, int64_t count) {
  if (T->nnode == T->cap) {
    T->cap = T->cap ? 2 * T->cap : 64;
    T->depth = realloc(T->depth, sizeof(int) * T->cap);
    T->parent = realloc(T->parent, sizeof(int) * T->cap);
    T->coord = realloc(T->coord, sizeof(int) * 3 * T->cap);
    T->start = realloc(T->start, sizeof(int64_t) * T->cap);
    T->count = realloc(T->count, sizeof(int64_t) * T->cap);
  }
  int id = T->nnode++;
  T->depth[id] = depth;
  T->parent[id] = parent;
  for (int d = 0; d < 3; d++) T->coord[3 * id + d] = coord[d];
  T->start[id] = start;
  T->count[id] = count;
  if (depth > T->maxdepth) T->maxdepth = depth;
  return id;
}

/* Stable partition of idx[start, start+count) into the 2^d children, then
 * recursion in child order (pre-order numbering). */
static void split(otree *T, const double *pts, int64_t *idx, int64_t *tmp, int node) {
  int64_t s = T->start[node], c = T->count[node];
  int t = T->depth[node];
  if (c <= T->leaf || t >= 20) return;
  int nch = 1 << T->dim;
  int64_t cnt[8] = {0};
  for (int64_t q = s; q < s + c; q++) {
    const double *p = pts + idx[q] * T->dim;
    int ch = 0;
    for (int d = 0; d < T->dim; d++) ch |= (int)(cellc(p[d], t + 1) & 1) << d;
    cnt[ch]++;
  }
  int64_t off[8] = {0};
  int64_t acc = s;
  for (int ch = 0; ch < nch; ch++) {
    off[ch] = acc;
    acc += cnt[ch];
  }
  int64_t pos[8];
  memcpy(pos, off, sizeof(pos));
  for (int64_t q = s; q < s + c; q++) {
    const double *p = pts + idx[q] * T->dim;
    int ch = 0;
    for (int d = 0; d < T->dim; d++) ch |= (int)(cellc(p[d], t + 1) & 1) << d;
    tmp[pos[ch]++] = idx[q];
  }
  memcpy(idx + s, tmp + s, sizeof(int64_t) * c);
  for (int ch = 0; ch < nch; ch++) {
    if (cnt[ch] == 0) continue;
    int cc[3] = {0, 0, 0};
    for (int d = 0; d < T->dim; d++) cc[d] = 2 * T->coord[3 * node + d] + ((ch >> d) & 1);
    int id = new_node(T, t + 1, node, cc, off[ch], cnt[ch]);
    split(T, pts, idx, tmp, id);
  }
}

void *orc_tree_build(const double *pts, int64_t n, int dim, int leaf) {
  if (n < 0 || (dim != 2 && dim != 3) || leaf < 1) return NULL;
  otree *T = calloc(1, sizeof(otree));
  T->dim = dim;
  T->leaf = leaf;
  T->n = n;
  T->perm = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  int64_t *tmp = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  for (int64_t i = 0; i < n; i++) T->perm[i] = i;
  int zero[3] = {0, 0, 0};
  int root = new_node(T, 0, -1, zero, 0, n);
  split(T, pts, T->perm, tmp, root);
  free(tmp);
  T->x = malloc(sizeof(double) * dim * (n > 0 ? n : 1));
  for (int64_t g = 0; g < n; g++)
    for (int d = 0; d < dim; d++) T->x[g * dim + d] = pts[T->perm[g] * dim + d];
  return T;
}

void orc_tree_free(void *h) {
  otree *T = h;
  if (!T) return;
  free(T->perm); free(T->x); free(T->depth); free(T->parent);
  free(T->coord); free(T->start); free(T->count);
  free(T);
}

/* what: 0 nnode, 1 maxdepth, 2 n, 3 dim */
int64_t orc_tree_info(void *h, int what) {
  otree *T = h;
  switch (what) {
    case 0: return T->nnode;
    case 1: return T->maxdepth;
    case 2: return T->n;
    case 3: return T->dim;
  }
  return -1;
}

void orc_tree_perm(void *h, int64_t *perm) {
  otree *T = h;
  memcpy(perm, T->perm, sizeof(int64_t) * T->n);
}

void orc_tree_nodes(void *h, int *depth, int *parent, int *coord3, int64_t *start, int64_t *count) {
  otree *T = h;
  memcpy(depth, T->depth, sizeof(int) * T->nnode);
  memcpy(parent, T->parent, sizeof(int) * T->nnode);
  memcpy(coord3, T->coord, sizeof(int) * 3 * T->nnode);
  memcpy(start, T->start, sizeof(int64_t) * T->nnode);
  memcpy(count, T->count, sizeof(int64_t) * T->nnode);
}

static uint64_t morton(const int *c, int dim) {
  uint64_t m = 0;
  for (int b = 0; b < 21; b++)
    for (int d = 0; d < dim; d++) m |= (uint64_t)((c[d] >> b) & 1) << (dim * b + d);
  return m;
}

/* Colour of a cell: sum_d (c_d mod base) base^d; base 3 (the boxes of a
 * colour are >= 3 cells apart) except while a factorization with the 2^d
 * schedule orders its levels. */
static int g_colour_base = 3;
static int colour(const int *c, int dim) {
  int col = 0, mul = 1;
  for (int d = 0; d < dim; d++) {
    col += (c[d] % g_colour_base) * mul;
    mul *= g_colour_base;
  }
  return col;
}

static const otree *g_sort_tree;
static int cmp_box(const void *a, const void *b) {
  const otree *T = g_sort_tree;
  int i = *(const int *)a, j = *(const int *)b;
  int ci = colour(T->coord + 3 * i, T->dim), cj = colour(T->coord + 3 * j, T->dim);
  if (ci != cj) return ci < cj ? -1 : 1;
  uint64_t mi = morton(T->coord + 3 * i, T->dim), mj = morton(T->coord + 3 * j, T->dim);
  if (mi != mj) return mi < mj ? -1 : 1;
  return 0;
}

/* Boxes of depth t in elimination order; returns the count. */
int orc_tree_level_boxes(void *h, int t, int *out) {
  otree *T = h;
  int nb = 0;
  for (int i = 0; i < T->nnode; i++)
    if (T->depth[i] == t) out[nb++] = i;
  g_sort_tree = T;
  qsort(out, nb, sizeof(int), cmp_box);
  return nb;
}

static int cheb(const int64_t *a, const int64_t *b, int dim) {
  int64_t m = 0;
  for (int d = 0; d < dim; d++) {
    int64_t z = a[d] - b[d];
    if (z < 0) z = -z;
    if (z > m) m = z;
  }
  return m > 1000000 ? 1000000 : (int)m;
}

/* Depth-t cells of all points (tree order), 3 per point. */
static int64_t *cells_at(const otree *T, int t) {
  int64_t *c = calloc((size_t)3 * (T->n > 0 ? T->n : 1), sizeof(int64_t));
  for (int64_t g = 0; g < T->n; g++)
    for (int d = 0; d < T->dim; d++) c[3 * g + d] = cellc(T->x[g * T->dim + d], t);
  return c;
}

/* Neighbour cells of node `node` that hold at least one point at the node's
 * depth, as offset codes sum_d (delta_d + 2) 5^d; near (distance 1) and ring
 * (distance 2) separately, ascending.  Brute force over all points. */
int orc_tree_box_lists(void *h, int node, int *near, int *nnear, int *ring, int *nring) {
  otree *T = h;
  int t = T->depth[node];
  int ncode = T->dim == 2 ? 25 : 125;
  int seen[125];
  memset(seen, 0, sizeof(seen));
  int64_t bc[3] = {T->coord[3 * node], T->coord[3 * node + 1], T->coord[3 * node + 2]};
  for (int64_t g = 0; g < T->n; g++) {
    int64_t c[3] = {0, 0, 0};
    for (int d = 0; d < T->dim; d++) c[d] = cellc(T->x[g * T->dim + d], t);
    int dist = cheb(c, bc, T->dim);
    if (dist < 1 || dist > 2) continue;
    int code = 0, mul = 1;
    for (int d = 0; d < T->dim; d++) {
      code += (int)(c[d] - bc[d] + 2) * mul;
      mul *= 5;
    }
    seen[code] = dist;
  }
  *nnear = 0;
  *nring = 0;
  for (int code = 0; code < ncode; code++) {
    if (seen[code] == 1) near[(*nnear)++] = code;
    if (seen[code] == 2) ring[(*nring)++] = code;
  }
  return 0;
}

/* Mistakes planted on purpose by the tests, to show whether a check catches
 * them: 0 none; 1 every proxy surface centred one box side off in x; 2 the
 * strong ID matrix holds only the ring cells at x offset >= 0 (the wrong
 * ring cells); 3 the proxy radius a quarter of the one asked for (a circle
 * through the box itself); 4 the ID takes its pivots in column order
 * (no pivoting). */
static int g_plant = 0;
void orc_plant_mistake(int what) { g_plant = what; }

/* ------------------------------------------------------------------------ */
/* Dense building blocks                                                      */
/* ------------------------------------------------------------------------ */

/* Interpolative decomposition of M (m x n, column-major, overwritten) by
 * Householder QR with greedy column pivoting (Definition 2.1 and the remark
 * after it).  perm: n entries, first k skeleton columns in pivot order, then
 * the redundant ones.  T: k x (n-k), column-major (ld k), T = R11^{-1} R12.
 * rdiag: |R_jj| for j < min(m,n) steps taken (may be NULL).  Returns k. */
int orc_cpqr_id(double *M, int m, int n, double eps, int *perm, double *T, double *rdiag) {
  for (int j = 0; j < n; j++) perm[j] = j;
  int steps = m < n ? m : n;
  double *nrm = malloc(sizeof(double) * (n > 0 ? n : 1));
  double *v = malloc(sizeof(double) * (m > 0 ? m : 1));
  double r11 = 0.0;
  int k = 0;
  for (int j = 0; j < steps; j++) {
    /* trailing column norms, recomputed */
    int p = j;
    double best = -1.0;
    for (int c = j; c < n; c++) {
      double s = 0.0;
      for (int i = j; i < m; i++) s += M[(size_t)c * m + i] * M[(size_t)c * m + i];
      nrm[c] = s;
      if (s > best) {
        best = s;
        p = c;
      }
    }
    if (g_plant == 4) best = nrm[p = j];
    double colnorm = sqrt(best);
    if (j == 0) r11 = colnorm;
    if (rdiag) rdiag[j] = colnorm;
    if (r11 == 0.0 || !(colnorm > eps * r11)) break;
    /* swap columns j and p */
    if (p != j) {
      for (int i = 0; i < m; i++) {
        double tmp = M[(size_t)j * m + i];
        M[(size_t)j * m + i] = M[(size_t)p * m + i];
        M[(size_t)p * m + i] = tmp;
      }
      int tp = perm[j];
      perm[j] = perm[p];
      perm[p] = tp;
    }
    /* Householder reflector H = I - 2 v v^T / (v^T v) mapping x -> alpha e1 */
    double *x = M + (size_t)j * m;
    double alpha = x[j] >= 0.0 ? -colnorm : colnorm;
    double vv = 0.0;
    for (int i = j; i < m; i++) v[i] = x[i];
    v[j] -= alpha;
    for (int i = j; i < m; i++) vv += v[i] * v[i];
    if (vv > 0.0) {
      for (int c = j + 1; c < n; c++) {
        double *y = M + (size_t)c * m;
        double s = 0.0;
        for (int i = j; i < m; i++) s += v[i] * y[i];
        double f = 2.0 * s / vv;
        for (int i = j; i < m; i++) y[i] -= f * v[i];
      }
    }
    x[j] = alpha;
    for (int i = j + 1; i < m; i++) x[i] = 0.0;
    k = j + 1;
  }
  /* T = R11^{-1} R12 by back substitution, column by column */
  int r = n - k;
  for (int c = 0; c < r; c++) {
    for (int i = k - 1; i >= 0; i--) {
      double s = M[(size_t)(k + c) * m + i];
      for (int l = i + 1; l < k; l++) s -= M[(size_t)l * m + i] * T[(size_t)c * k + l];
      T[(size_t)c * k + i] = s / M[(size_t)i * m + i];
    }
  }
  free(nrm);
  free(v);
  return k;
}

/* LU with partial pivoting of A (n x n, row-major, overwritten with L\U):
 * row i of P A is row piv[i] of A; P A = L U.  Pivot = largest |entry| in
 * the column, ties to the lowest row.  Returns 0, or j+1 if pivot j is 0. */
int orc_lu(double *A, int n, int *piv) {
  int info = 0;
  for (int i = 0; i < n; i++) piv[i] = i;
  for (int j = 0; j < n; j++) {
    int p = j;
    double best = fabs(A[(size_t)j * n + j]);
    for (int i = j + 1; i < n; i++) {
      double a = fabs(A[(size_t)i * n + j]);
      if (a > best) {
        best = a;
        p = i;
      }
    }
    if (p != j) {
      for (int c = 0; c < n; c++) {
        double tmp = A[(size_t)j * n + c];
        A[(size_t)j * n + c] = A[(size_t)p * n + c];
        A[(size_t)p * n + c] = tmp;
      }
      int tp = piv[j];
      piv[j] = piv[p];
      piv[p] = tp;
    }
    double d = A[(size_t)j * n + j];
    if (d == 0.0) {
      if (!info) info = j + 1;
      continue;
    }
    for (int i = j + 1; i < n; i++) {
      double l = A[(size_t)i * n + j] / d;
      A[(size_t)i * n + j] = l;
      for (int c = j + 1; c < n; c++) A[(size_t)i * n + c] -= l * A[(size_t)j * n + c];
    }
  }
  return info;
}

/* Cholesky X = L L^T of a symmetric positive definite X (n x n, row-major,
 * symmetric part used), stored in the LU layout so that every LU routine
 * applies it: unit lower L D^{-1} below the diagonal, U = D L^T on and above
 * it (D = diag(L)), identity pivots.  Returns 0, or j+1 if the leading
 * block of order j+1 is not positive definite. */
static int chol_as_lu(double *X, int n, int *piv) {
  for (int i = 0; i < n; i++) piv[i] = i;  /* valid even when it fails */
  double *L = calloc((size_t)n * n + 1, sizeof(double));
  for (int j = 0; j < n; j++) {
    double d = X[(size_t)j * n + j];
    for (int l = 0; l < j; l++) d -= L[(size_t)j * n + l] * L[(size_t)j * n + l];
    if (!(d > 0.0)) {
      free(L);
      return j + 1;
    }
    L[(size_t)j * n + j] = sqrt(d);
    for (int i = j + 1; i < n; i++) {
      double s = 0.5 * (X[(size_t)i * n + j] + X[(size_t)j * n + i]);
      for (int l = 0; l < j; l++) s -= L[(size_t)i * n + l] * L[(size_t)j * n + l];
      L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
    }
  }
  for (int i = 0; i < n; i++) {
    for (int j = 0; j < n; j++)
      X[(size_t)i * n + j] = i > j ? L[(size_t)i * n + j] / L[(size_t)j * n + j]
                                   : L[(size_t)j * n + i] * L[(size_t)i * n + i];
  }
  free(L);
  return 0;
}

/* Solve (P^T L U) X = B for X, B n x nrhs column-major (overwritten). */
static void lu_solve(const double *LU, const int *piv, int n, double *B, int nrhs) {
  double *y = malloc(sizeof(double) * (n > 0 ? n : 1));
  for (int c = 0; c < nrhs; c++) {
    double *b = B + (size_t)c * n;
    for (int i = 0; i < n; i++) y[i] = b[piv[i]];
    for (int i = 0; i < n; i++)
      for (int l = 0; l < i; l++) y[i] -= LU[(size_t)i * n + l] * y[l];
    for (int i = n - 1; i >= 0; i--) {
      for (int l = i + 1; l < n; l++) y[i] -= LU[(size_t)i * n + l] * y[l];
      y[i] /= LU[(size_t)i * n + i];
    }
    memcpy(b, y, sizeof(double) * n);
  }
  free(y);
}

/* Solve X (P^T L U) = B for X, B nr x n row-major (overwritten):
 * X P^T L U = B;  with Z = X P^T:  (Z L) U = B.  */
static void lu_solve_right(const double *LU, const int *piv, int n, double *B, int nr) {
  double *w = malloc(sizeof(double) * (n > 0 ? n : 1));
  for (int q = 0; q < nr; q++) {
    double *b = B + (size_t)q * n;
    /* W U = b  (forward over columns) */
    for (int j = 0; j < n; j++) {
      double s = b[j];
      for (int i = 0; i < j; i++) s -= w[i] * LU[(size_t)i * n + j];
      w[j] = s / LU[(size_t)j * n + j];
    }
    /* Z L = W, L unit lower (backward over columns) */
    for (int j = n - 1; j >= 0; j--) {
      double s = w[j];
      for (int i = j + 1; i < n; i++) s -= b[i] * LU[(size_t)i * n + j];
      b[j] = s; /* b now holds Z entries from j on */
    }
    /* X = Z P: X[:, piv[i]] = Z[:, i] */
    for (int i = 0; i < n; i++) w[piv[i]] = b[i];
    memcpy(b, w, sizeof(double) * n);
  }
  free(w);
}

/* y = (P^T L U) x for n x nrhs column-major. */
static void lu_mult(const double *LU, const int *piv, int n, const double *x, double *y, int nrhs) {
  double *u = malloc(sizeof(double) * (n > 0 ? n : 1));
  for (int c = 0; c < nrhs; c++) {
    const double *xc = x + (size_t)c * n;
    for (int i = 0; i < n; i++) {
      double s = 0.0;
      for (int l = i; l < n; l++) s += LU[(size_t)i * n + l] * xc[l];
      u[i] = s;
    }
    double *yc = y + (size_t)c * n;
    for (int i = 0; i < n; i++) {
      double s = u[i];
      for (int l = 0; l < i; l++) s += LU[(size_t)i * n + l] * u[l];
      yc[piv[i]] = s;
    }
  }
  free(u);
}

/* ------------------------------------------------------------------------ */
/* RS-S factorization (Algorithm 1)                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
  int node, depth, b, k, r, nj, nnear, nring;
  int weak;           /* 1: weak skeletonization (RS-WS, Sec. 3.4): J = S */
  int64_t *S, *R, *J; /* tree-order DOF ids: S in pivot order, J = [S; N] */
  double *T;          /* k x r column-major (ld k) */
  double *LU;         /* r x r row-major */
  int *piv;
  double *E; /* nj x r row-major:  E = X_JR X_RR^{-1} */
  double *G; /* r x nj row-major:  G = X_RR^{-1} X_RJ */
} obox;

typedef struct {
  const otree *T;
  okern kn;
  double eps;
  int nbox;
  obox *box;
  int ntop;
  int64_t *top;
  double *LUtop;
  int *pivtop;
  double **chol;      /* Cholesky factors of the X_RR blocks and the top (orc_sqrt_prepare) */
  int64_t violations; /* Theorem 3.1 / Corollary 3.2 violations seen */
  int info;           /* nonzero: zero pivot met */
  /* per-box ID checks (check mode): boxes whose ID residual exceeds the
   * column-pivoted QR bound, boxes whose T fails to compress the full far
   * field to 10 eps, and the worst ratio of each (residual / bound) */
  int64_t id_violations, proxy_violations;
  double id_worst, proxy_worst;
} ofactor;



static void proxy_points(int dim, int np, double radius, int t, const int *coord, double *y) {
  double D = ldexp(1.0, -t);
  double c[3];
  for (int d = 0; d < dim; d++) c[d] = (coord[d] + 0.5) * D;
  if (g_plant == 1) c[0] += D;
  if (g_plant == 3) radius *= 0.25;
  for (int m = 0; m < np; m++) {
    if (dim == 2) {
      double th = 2.0 * ORC_PI * (double)m / (double)np;
      y[2 * m] = c[0] + radius * D * cos(th);
      y[2 * m + 1] = c[1] + radius * D * sin(th);
    } else {
      double z = 1.0 - (2.0 * m + 1.0) / (double)np;
      double rr = sqrt(1.0 - z * z);
      double ph = (double)m * ORC_PI * (3.0 - sqrt(5.0));
      y[3 * m] = c[0] + radius * D * rr * cos(ph);
      y[3 * m + 1] = c[1] + radius * D * rr * sin(ph);
      y[3 * m + 2] = c[2] + radius * D * z;
    }
  }
}

/* Residual X[:, R] - X[:, S] T of an ID with the columns of X (mx x b,
 * column-major) taken in the order perm (S = perm[0..k), R = perm[k..b)),
 * T k x r column-major: returns it as an mx x r column-major array. */
static double *id_residual(const double *X, int64_t mx, int b, const int *perm, int k, const double *T) {
  int r = b - k;
  double *Res = malloc(sizeof(double) * ((size_t)mx * r + 1));
  for (int c = 0; c < r; c++) {
    const double *xr = X + (size_t)perm[k + c] * mx;
    double *o = Res + (size_t)c * mx;
    for (int64_t i = 0; i < mx; i++) o[i] = xr[i];
    for (int s = 0; s < k; s++) {
      double t = T[(size_t)c * k + s];
      const double *xs = X + (size_t)perm[s] * mx;
      for (int64_t i = 0; i < mx; i++) o[i] -= xs[i] * t;
    }
  }
  return Res;
}

static double fro(const double *X, size_t len) {
  double s = 0.0;
  for (size_t i = 0; i < len; i++) s += X[i] * X[i];
  return sqrt(s);
}

/* ||X||_2 of X (mx x nc, column-major): power iteration on X^T X (a lower
 * estimate that converges to the largest singular value). */
static double norm2(const double *X, int64_t mx, int nc) {
  if (nc == 0 || mx == 0) return 0.0;
  double *G = calloc((size_t)nc * nc, sizeof(double));
  for (int a = 0; a < nc; a++)
    for (int c = a; c < nc; c++) {
      double s = 0.0;
      for (int64_t i = 0; i < mx; i++) s += X[(size_t)a * mx + i] * X[(size_t)c * mx + i];
      G[(size_t)a * nc + c] = G[(size_t)c * nc + a] = s;
    }
  double *v = malloc(sizeof(double) * nc), *u = malloc(sizeof(double) * nc);
  for (int a = 0; a < nc; a++) v[a] = 1.0 + 0.01 * (a % 7);
  double lam = 0.0;
  for (int it = 0; it < 300; it++) {
    double nv = 0.0;
    for (int a = 0; a < nc; a++) nv += v[a] * v[a];
    nv = sqrt(nv);
    if (nv == 0.0) break;
    for (int a = 0; a < nc; a++) v[a] /= nv;
    double q = 0.0;
    for (int a = 0; a < nc; a++) {
      double s = 0.0;
      for (int c = 0; c < nc; c++) s += G[(size_t)a * nc + c] * v[c];
      u[a] = s;
      q += v[a] * s;
    }
    lam = q > lam ? q : lam;
    memcpy(v, u, sizeof(double) * nc);
  }
  free(G); free(v); free(u);
  return sqrt(lam > 0.0 ? lam : 0.0);
}

/* Factor.  check != 0 turns on the Theorem 3.1 / Corollary 3.2 checks and
 * two checks of every box's ID (Definition 2.1, Sec. 3.2):
 *   - the column-pivoted QR bound on the ID matrix M the box formed: every
 *     trailing column of R after k steps has norm <= |R_kk+1| <= eps |R_11|,
 *     so ||M_R - M_S T||_F <= sqrt(r) eps |R_11| (up to rounding);
 *   - proxy validity: the same T compresses the box's interactions with its
 *     whole far field F (every active DOF at distance >= 2, the ring O and
 *     the rest P), ||X_R - X_S T||_2 <= 10 eps ||X||_2 for
 *     X = [A_FB; A_BF^T] from the current matrix.
 * schedule: 0 one box after another in colour order (3^d colours); 1 and 2
 * a colour phase as a parallel machine runs it, with 3^d (1) or 2^d (2)
 * colours (Sec. 5): every box of the phase builds its lists and its ID
 * matrix from the state at the start of the phase.  The rest of a box's
 * step reads only its own rows / columns and its neighbours', which no
 * other box of the phase writes except through the additive Schur updates
 * of shared near-field blocks, so running those parts one box after
 * another equals the parallel phase up to the order of those additions.
 * With 3^d colours no box of a phase is within two cells of another, so
 * schedule 1 gives the same factor as schedule 0.
 * hybrid != 0: RS-WS (Sec. 3.4, Algorithm 2): at every depth, first weak
 * skeletonization of each box (its interactions with the whole complement
 * compressed: the cells inside the proxy surface explicitly, the rest
 * through the proxy points), then strong skeletonization of what stays
 * active; plus a last weak pass at depth 1, where no strong step is
 * possible, as the paper does in practice. */
void *orc_factor(void *th, int kind, double diag, double w, double eps, int nproxy,
                 double radius, int check, int hybrid, int schedule, int chol) {
  otree *T = th;
  int64_t n = T->n;
  int dim = T->dim;
  ofactor *F = calloc(1, sizeof(ofactor));
  F->T = T;
  F->kn.kind = kind;
  F->kn.dim = dim;
  F->kn.diag = diag;
  F->kn.w = w;
  F->eps = eps;
  if (nproxy <= 0) nproxy = dim == 2 ? 64 : 512;
  if (radius <= 0.0) radius = 2.5;

  /* A := K (the full matrix, row-major) */
  double *A = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = 0; j < n; j++) A[i * n + j] = entry(&F->kn, T->x, i, j);
  char *active = malloc(n > 0 ? n : 1);
  memset(active, 1, n > 0 ? n : 1);

  int64_t *Bl = malloc(sizeof(int64_t) * (n + 1)), *Nl = malloc(sizeof(int64_t) * (n + 1));
  int64_t *Ol = malloc(sizeof(int64_t) * (n + 1)), *Pl = malloc(sizeof(int64_t) * (n + 1));
  int *order = malloc(sizeof(int) * (T->nnode + 1));
  double *yp = malloc(sizeof(double) * 3 * nproxy);
  int cap = 16;
  F->box = malloc(sizeof(obox) * cap);
  /* phase-start state for the parallel schedules */
  double *A0 = schedule ? malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1)) : NULL;
  char *active0 = schedule ? malloc(n > 0 ? n : 1) : NULL;

  for (int t = T->maxdepth; t >= (hybrid ? 1 : 2); t--) {
    int64_t *cell = cells_at(T, t);
    g_colour_base = schedule == 2 ? 2 : 3;
    int nb = orc_tree_level_boxes(T, t, order);
    g_colour_base = 3;
    if (check) {
      /* Corollary 3.2: at the start of a level, every far-field entry of
       * every box of this level equals the original kernel entry. */
      for (int q = 0; q < nb; q++) {
        int node = order[q];
        int64_t bc[3] = {T->coord[3 * node], T->coord[3 * node + 1], T->coord[3 * node + 2]};
        for (int64_t i = T->start[node]; i < T->start[node] + T->count[node]; i++) {
          if (!active[i]) continue;
          for (int64_t j = 0; j < n; j++) {
            if (!active[j] || cheb(cell + 3 * j, bc, dim) < 2) continue;
            if (A[i * n + j] != entry(&F->kn, T->x, i, j)) F->violations++;
            if (A[j * n + i] != entry(&F->kn, T->x, j, i)) F->violations++;
          }
        }
      }
    }
    /* pass 0: weak skeletonization (RS-WS only); pass 1: strong (depths >= 2) */
    for (int pass = hybrid ? 0 : 1; pass <= (t >= 2 ? 1 : 0); pass++) {
    const int weak = pass == 0;
    for (int q = 0; q < nb; q++) {
      int node = order[q];
      int64_t bc[3] = {T->coord[3 * node], T->coord[3 * node + 1], T->coord[3 * node + 2]};
      /* parallel schedules: the state at the start of the colour phase */
      const int par = schedule && !weak;
      if (par) {
        const int base = schedule == 2 ? 2 : 3;
        int newphase = q == 0;
        if (!newphase) {
          g_colour_base = base;
          newphase = colour(T->coord + 3 * node, dim) != colour(T->coord + 3 * order[q - 1], dim);
          g_colour_base = 3;
        }
        if (newphase) {
          memcpy(A0, A, sizeof(double) * (size_t)n * (size_t)n);
          memcpy(active0, active, (size_t)n);
        }
      }
      const double *Ar = par ? A0 : A;
      const char *act = par ? active0 : active;
      /* B: active DOFs of the box; N / O / P by cell distance (Fig. 2) */
      int64_t nbB = 0, nN = 0, nO = 0, nP = 0;
      for (int64_t g = T->start[node]; g < T->start[node] + T->count[node]; g++)
        if (act[g]) Bl[nbB++] = g;
      for (int64_t g = 0; g < n; g++) {
        if (!act[g]) continue;
        int dist = cheb(cell + 3 * g, bc, dim);
        if (dist == 1) Nl[nN++] = g;
        else if (dist == 2) Ol[nO++] = g;
        else if (dist >= 3) Pl[nP++] = g;
      }
      if (nbB == 0) continue;
      if (check) {
        /* Theorem 3.1: interactions between B and P are still original (P
         * DOFs eliminated earlier in a parallel phase are decoupled, not
         * part of the remaining matrix) */
        for (int64_t a = 0; a < nbB; a++)
          for (int64_t p = 0; p < nP; p++) {
            int64_t i = Bl[a], j = Pl[p];
            if (!active[j]) continue;
            if (A[i * n + j] != entry(&F->kn, T->x, i, j)) F->violations++;
            if (A[j * n + i] != entry(&F->kn, T->x, j, i)) F->violations++;
          }
      }
      int b = (int)nbB;
      /* ID matrix [A_XB; A_BX^T; w K(Gamma,B); w K(B,Gamma)^T], column-major,
       * with X the cells inside the proxy surface that the step compresses:
       * strong: the ring O (Eq. 3.7); weak: N and O (the whole complement) */
      int64_t nX = weak ? nN + nO : nO;
      /* planted mistake 2 (tests only): part of the ring left out */
      int64_t *Om = Ol;
      if (g_plant == 2 && !weak) {
        Om = malloc(sizeof(int64_t) * (nO + 1));
        nX = 0;
        for (int64_t o = 0; o < nO; o++)
          if (cell[3 * Ol[o]] >= bc[0]) Om[nX++] = Ol[o];
      }
      int m = (int)(2 * nX + 2 * nproxy);
      double *M = malloc(sizeof(double) * (size_t)m * b);
      proxy_points(dim, nproxy, radius, t, T->coord + 3 * node, yp);
      for (int c = 0; c < b; c++) {
        int64_t j = Bl[c];
        double *col = M + (size_t)c * m;
        for (int64_t o = 0; o < nX; o++) {
          int64_t g = weak && o < nN ? Nl[o] : Om[weak ? o - nN : o];
          col[o] = Ar[g * n + j];
          col[nX + o] = Ar[j * n + g];
        }
        for (int p = 0; p < nproxy; p++) {
          col[2 * nX + p] = w * kfun(kind, dim, yp + dim * p, T->x + j * dim);
          col[2 * nX + nproxy + p] = w * kfun(kind, dim, T->x + j * dim, yp + dim * p);
        }
      }
      int *perm = malloc(sizeof(int) * b);
      double *Tm = malloc(sizeof(double) * (size_t)b * b + 1);
      double *M0 = check ? malloc(sizeof(double) * ((size_t)m * b + 1)) : NULL;
      double *rd = malloc(sizeof(double) * (b + 1));
      if (M0) memcpy(M0, M, sizeof(double) * (size_t)m * b);
      int k = orc_cpqr_id(M, m, b, eps, perm, Tm, rd);
      free(M);
      if (Om != Ol) free(Om);
      int r = b - k;
      if (check && r > 0) {
        const double u = 2.220446049250313e-16;
        /* the CPQR bound on the matrix the ID was computed from */
        double *Res = id_residual(M0, m, b, perm, k, Tm);
        double res = fro(Res, (size_t)m * r);
        double tn = fro(Tm, (size_t)k * r);
        double bound = sqrt((double)r) * eps * rd[0] + 8.0 * (m + b) * u * fro(M0, (size_t)m * b) * (1.0 + tn);
        if (res > bound) F->id_violations++;
        if (bound > 0.0 && res / bound > F->id_worst) F->id_worst = res / bound;
        free(Res);
        /* proxy validity against the full far field (ring and beyond) */
        int64_t nF = weak ? nN + nO + nP : nO + nP;
        double *X = malloc(sizeof(double) * ((size_t)2 * nF * b + 1));
        for (int c = 0; c < b; c++) {
          int64_t j = Bl[c];
          double *col = X + (size_t)c * 2 * nF;
          int64_t o = 0;
          if (weak)
            for (int64_t a = 0; a < nN; a++, o++) col[o] = Ar[Nl[a] * n + j], col[nF + o] = Ar[j * n + Nl[a]];
          for (int64_t a = 0; a < nO; a++, o++) col[o] = Ar[Ol[a] * n + j], col[nF + o] = Ar[j * n + Ol[a]];
          for (int64_t a = 0; a < nP; a++, o++) col[o] = Ar[Pl[a] * n + j], col[nF + o] = Ar[j * n + Pl[a]];
        }
        if (nF > 0) {
          double *Rf = id_residual(X, 2 * nF, b, perm, k, Tm);
          double rf = norm2(Rf, 2 * nF, r), xf = norm2(X, 2 * nF, b);
          double pb = eps * xf + 8.0 * (2 * nF + b) * u * fro(X, (size_t)2 * nF * b) * (1.0 + tn);
          if (rf > pb) F->proxy_violations++;
          if (pb > 0.0 && rf / pb > F->proxy_worst) F->proxy_worst = rf / pb;
          free(Rf);
        }
        free(X);
      }
      free(M0);
      free(rd);

      if (F->nbox == cap) {
        cap *= 2;
        F->box = realloc(F->box, sizeof(obox) * cap);
      }
      obox *bx = &F->box[F->nbox++];
      memset(bx, 0, sizeof(obox));
      bx->node = node;
      bx->weak = weak;
      bx->depth = t;
      bx->b = b;
      bx->k = k;
      bx->r = r;
      bx->nnear = weak ? 0 : (int)nN;
      bx->nring = (int)nX;
      bx->S = malloc(sizeof(int64_t) * (k + 1));
      bx->R = malloc(sizeof(int64_t) * (r + 1));
      for (int i = 0; i < k; i++) bx->S[i] = Bl[perm[i]];
      for (int i = 0; i < r; i++) bx->R[i] = Bl[perm[k + i]];
      bx->T = malloc(sizeof(double) * ((size_t)k * r + 1));
      memcpy(bx->T, Tm, sizeof(double) * (size_t)k * r);
      free(Tm);
      free(perm);
      int64_t *S = bx->S, *R = bx->R;

      /* C: the rows / columns the operators U_T, L_T touch, B u N (strong);
       * B (weak: R's couplings outside the box are dropped below) */
      int64_t nC = weak ? nbB : nbB + nN;
      int64_t *C = malloc(sizeof(int64_t) * (nC + 1));
      memcpy(C, Bl, sizeof(int64_t) * nbB);
      if (!weak) memcpy(C + nbB, Nl, sizeof(int64_t) * nN);
      const double *Tk = bx->T;
      /* U_T from the left: rows R -= T^T rows S (Sec. 3.1) */
      for (int ri = 0; ri < r; ri++)
        for (int64_t c = 0; c < nC; c++) {
          double s = 0.0;
          for (int si = 0; si < k; si++) s += Tk[(size_t)ri * k + si] * A[S[si] * n + C[c]];
          A[R[ri] * n + C[c]] -= s;
        }
      /* L_T from the right: columns R -= columns S T (Sec. 3.1) */
      for (int64_t c = 0; c < nC; c++)
        for (int ri = 0; ri < r; ri++) {
          double s = 0.0;
          for (int si = 0; si < k; si++) s += A[C[c] * n + S[si]] * Tk[(size_t)ri * k + si];
          A[C[c] * n + R[ri]] -= s;
        }
      /* The compressed blocks are dropped (set to 0): X_RF, X_FR for the far
       * field (strong), every coupling of R outside the box (weak). */
      for (int ri = 0; ri < r; ri++)
        for (int64_t g = 0; g < n; g++) {
          if (!active[g]) continue;
          int dist = cheb(cell + 3 * g, bc, dim);
          if (dist >= (weak ? 1 : 2)) {
            A[R[ri] * n + g] = 0.0;
            A[g * n + R[ri]] = 0.0;
          }
        }
      /* Block elimination with I = R, J = S u N (Sec. 2.1, Eq. 3.4); J = S
       * after a weak step */
      int nj = (int)(weak ? k : k + nN);
      bx->nj = nj;
      bx->J = malloc(sizeof(int64_t) * (nj + 1));
      memcpy(bx->J, S, sizeof(int64_t) * k);
      if (!weak) memcpy(bx->J + k, Nl, sizeof(int64_t) * nN);
      int64_t *J = bx->J;
      bx->LU = malloc(sizeof(double) * ((size_t)r * r + 1));
      bx->piv = malloc(sizeof(int) * (r + 1));
      for (int i = 0; i < r; i++)
        for (int j = 0; j < r; j++) bx->LU[(size_t)i * r + j] = A[R[i] * n + R[j]];
      /* LU with partial pivoting, or Cholesky for positive definite K
       * (Sec. 4: the paper's choice for its diagonal blocks) */
      int info = chol ? chol_as_lu(bx->LU, r, bx->piv) : orc_lu(bx->LU, r, bx->piv);
      if (info && !F->info) F->info = info;
      bx->E = malloc(sizeof(double) * ((size_t)nj * r + 1));
      bx->G = malloc(sizeof(double) * ((size_t)r * nj + 1));
      for (int a = 0; a < nj; a++)
        for (int ri = 0; ri < r; ri++) bx->E[(size_t)a * r + ri] = A[J[a] * n + R[ri]];
      lu_solve_right(bx->LU, bx->piv, r, bx->E, nj);
      if (chol) {
        /* symmetric K: G = E^T (Sec. 3.3.3, V_i = W_i^T); only E is needed */
        for (int ri = 0; ri < r; ri++)
          for (int a = 0; a < nj; a++) bx->G[(size_t)ri * nj + a] = bx->E[(size_t)a * r + ri];
      } else {
        /* G column-major scratch (r x nj), then stored row-major */
        double *Gc = malloc(sizeof(double) * ((size_t)r * nj + 1));
        for (int a = 0; a < nj; a++)
          for (int ri = 0; ri < r; ri++) Gc[(size_t)a * r + ri] = A[R[ri] * n + J[a]];
        lu_solve(bx->LU, bx->piv, r, Gc, nj);
        for (int ri = 0; ri < r; ri++)
          for (int a = 0; a < nj; a++) bx->G[(size_t)ri * nj + a] = Gc[(size_t)a * r + ri];
        free(Gc);
      }
      /* Schur complement A_JJ -= E A_RJ, then decouple R */
      for (int a = 0; a < nj; a++)
        for (int c = 0; c < nj; c++) {
          double s = 0.0;
          for (int ri = 0; ri < r; ri++) s += bx->E[(size_t)a * r + ri] * A[R[ri] * n + J[c]];
          A[J[a] * n + J[c]] -= s;
        }
      for (int ri = 0; ri < r; ri++)
        for (int a = 0; a < nj; a++) {
          A[R[ri] * n + J[a]] = 0.0;
          A[J[a] * n + R[ri]] = 0.0;
        }
      for (int ri = 0; ri < r; ri++) active[R[ri]] = 0;
      free(C);
    }
    }
    free(cell);
  }

  /* Top block: all remaining active DOFs (Sec. 3.3.3), factored by LU */
  int64_t nt = 0;
  for (int64_t g = 0; g < n; g++)
    if (active[g]) nt++;
  F->ntop = (int)nt;
  F->top = malloc(sizeof(int64_t) * (nt + 1));
  nt = 0;
  for (int64_t g = 0; g < n; g++)
    if (active[g]) F->top[nt++] = g;
  F->LUtop = malloc(sizeof(double) * ((size_t)nt * nt + 1));
  F->pivtop = malloc(sizeof(int) * (nt + 1));
  for (int64_t i = 0; i < nt; i++)
    for (int64_t j = 0; j < nt; j++) F->LUtop[i * nt + j] = A[F->top[i] * n + F->top[j]];
  int info = chol ? chol_as_lu(F->LUtop, (int)nt, F->pivtop) : orc_lu(F->LUtop, (int)nt, F->pivtop);
  if (info && !F->info) F->info = info;

  if (check) {
    /* After the last level the matrix is block diagonal with blocks R_i and
     * the top set (Sec. 3.3.3): count nonzeros coupling different blocks. */
    int *blk = malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int64_t g = 0; g < n; g++) blk[g] = -1;
    for (int i = 0; i < F->nbox; i++)
      for (int ri = 0; ri < F->box[i].r; ri++) blk[F->box[i].R[ri]] = i;
    for (int64_t i = 0; i < n; i++)
      for (int64_t j = 0; j < n; j++)
        if (blk[i] != blk[j] && A[i * n + j] != 0.0) F->violations++;
    free(blk);
  }

  free(A); free(active); free(Bl); free(Nl); free(Ol); free(Pl); free(order); free(yp);
  free(A0); free(active0);
  return F;
}

void orc_factor_free(void *h) {
  ofactor *F = h;
  if (!F) return;
  for (int i = 0; i < F->nbox; i++) {
    obox *b = &F->box[i];
    free(b->S); free(b->R); free(b->J); free(b->T); free(b->LU); free(b->piv);
    free(b->E); free(b->G);
  }
  if (F->chol) {
    for (int i = 0; i <= F->nbox; i++) free(F->chol[i]);
    free(F->chol);
  }
  free(F->box); free(F->top); free(F->LUtop); free(F->pivtop);
  free(F);
}

/* what: 0 nbox, 1 ntop, 2 violations, 3 info, 4 boxes over the CPQR ID
 * bound, 5 boxes failing proxy validity (check mode) */
int64_t orc_factor_info(void *h, int what) {
  ofactor *F = h;
  switch (what) {
    case 0: return F->nbox;
    case 1: return F->ntop;
    case 2: return F->violations;
    case 3: return F->info;
    case 4: return F->id_violations;
    case 5: return F->proxy_violations;
  }
  return -1;
}

/* info8 = {node, depth, b, k, r, nj, nnear, nring} */
void orc_factor_box(void *h, int i, int *info9) {
  ofactor *F = h;
  obox *b = &F->box[i];
  int v[9] = {b->node, b->depth, b->b, b->k, b->r, b->nj, b->nnear, b->nring, b->weak};
  memcpy(info9, v, sizeof(v));
}

/* Copies S (k), R (r), J (nj) ids and T (k x r col-major), E (nj x r row-major),
 * G (r x nj row-major); any pointer may be NULL. */
void orc_factor_box_data(void *h, int i, int64_t *S, int64_t *R, int64_t *J, double *T, double *E,
                         double *G) {
  ofactor *F = h;
  obox *b = &F->box[i];
  if (S) memcpy(S, b->S, sizeof(int64_t) * b->k);
  if (R) memcpy(R, b->R, sizeof(int64_t) * b->r);
  if (J) memcpy(J, b->J, sizeof(int64_t) * b->nj);
  if (T) memcpy(T, b->T, sizeof(double) * (size_t)b->k * b->r);
  if (E) memcpy(E, b->E, sizeof(double) * (size_t)b->nj * b->r);
  if (G) memcpy(G, b->G, sizeof(double) * (size_t)b->r * b->nj);
}

void orc_factor_top(void *h, int64_t *top) {
  ofactor *F = h;
  memcpy(top, F->top, sizeof(int64_t) * F->ntop);
}

/* log |det D| = sum of log |U_jj| over all diagonal blocks (Sec. 3.3.3). */
double orc_logdet(void *h) {
  ofactor *F = h;
  double s = 0.0;
  for (int i = 0; i < F->nbox; i++) {
    obox *b = &F->box[i];
    for (int j = 0; j < b->r; j++) s += log(fabs(b->LU[(size_t)j * b->r + j]));
  }
  for (int j = 0; j < F->ntop; j++) s += log(fabs(F->LUtop[(size_t)j * F->ntop + j]));
  return s;
}

/* Working vectors live in tree order, one column per right-hand side. */
static void to_tree(const ofactor *F, const double *x, double *v, int nrhs) {
  int64_t n = F->T->n;
  for (int c = 0; c < nrhs; c++)
    for (int64_t g = 0; g < n; g++) v[(size_t)c * n + g] = x[(size_t)c * n + F->T->perm[g]];
}
static void from_tree(const ofactor *F, const double *v, double *x, int nrhs) {
  int64_t n = F->T->n;
  for (int c = 0; c < nrhs; c++)
    for (int64_t g = 0; g < n; g++) x[(size_t)c * n + F->T->perm[g]] = v[(size_t)c * n + g];
}

/* y = F x (Eq. 3.10): W_1 .. W_n, then D, then V_n .. V_1.  x, y: n x nrhs
 * column-major in the caller's original point order. */
void orc_apply(void *h, const double *x, double *y, int nrhs) {
  ofactor *F = h;
  int64_t n = F->T->n;
  double *v = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * nrhs);
  double *u = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * nrhs);
  to_tree(F, x, v, nrhs);
  for (int c = 0; c < nrhs; c++) {
    double *vc = v + (size_t)c * n;
    for (int i = 0; i < F->nbox; i++) {
      obox *b = &F->box[i];
      /* L_T^{-1}: v_S += T v_R */
      for (int si = 0; si < b->k; si++) {
        double s = 0.0;
        for (int ri = 0; ri < b->r; ri++) s += b->T[(size_t)ri * b->k + si] * vc[b->R[ri]];
        vc[b->S[si]] += s;
      }
      /* U^{-1}: v_R += G v_J */
      for (int ri = 0; ri < b->r; ri++) {
        double s = 0.0;
        for (int a = 0; a < b->nj; a++) s += b->G[(size_t)ri * b->nj + a] * vc[b->J[a]];
        vc[b->R[ri]] += s;
      }
    }
  }
  /* D: diagonal blocks X_RR and the top block */
  memcpy(u, v, sizeof(double) * (size_t)n * nrhs);
  for (int c = 0; c < nrhs; c++) {
    double *vc = v + (size_t)c * n, *uc = u + (size_t)c * n;
    for (int i = 0; i < F->nbox; i++) {
      obox *b = &F->box[i];
      double *xi = malloc(sizeof(double) * (b->r + 1)), *yi = malloc(sizeof(double) * (b->r + 1));
      for (int ri = 0; ri < b->r; ri++) xi[ri] = vc[b->R[ri]];
      lu_mult(b->LU, b->piv, b->r, xi, yi, 1);
      for (int ri = 0; ri < b->r; ri++) uc[b->R[ri]] = yi[ri];
      free(xi);
      free(yi);
    }
    int nt = F->ntop;
    double *xt = malloc(sizeof(double) * (nt + 1)), *yt = malloc(sizeof(double) * (nt + 1));
    for (int i = 0; i < nt; i++) xt[i] = vc[F->top[i]];
    lu_mult(F->LUtop, F->pivtop, nt, xt, yt, 1);
    for (int i = 0; i < nt; i++) uc[F->top[i]] = yt[i];
    free(xt);
    free(yt);
    for (int i = F->nbox - 1; i >= 0; i--) {
      obox *b = &F->box[i];
      /* L^{-1}: u_J += E u_R */
      for (int a = 0; a < b->nj; a++) {
        double s = 0.0;
        for (int ri = 0; ri < b->r; ri++) s += b->E[(size_t)a * b->r + ri] * uc[b->R[ri]];
        uc[b->J[a]] += s;
      }
      /* U_T^{-1}: u_R += T^T u_S */
      for (int ri = 0; ri < b->r; ri++) {
        double s = 0.0;
        for (int si = 0; si < b->k; si++) s += b->T[(size_t)ri * b->k + si] * uc[b->S[si]];
        uc[b->R[ri]] += s;
      }
    }
  }
  from_tree(F, u, y, nrhs);
  free(v);
  free(u);
}

/* x = F^{-1} b (Eq. 3.11): V_1^{-1} .. V_n^{-1}, D^{-1}, W_n^{-1} .. W_1^{-1}. */
void orc_solve(void *h, const double *bvec, double *x, int nrhs) {
  ofactor *F = h;
  int64_t n = F->T->n;
  double *v = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * nrhs);
  to_tree(F, bvec, v, nrhs);
  for (int c = 0; c < nrhs; c++) {
    double *vc = v + (size_t)c * n;
    for (int i = 0; i < F->nbox; i++) {
      obox *b = &F->box[i];
      /* U_T: v_R -= T^T v_S */
      for (int ri = 0; ri < b->r; ri++) {
        double s = 0.0;
        for (int si = 0; si < b->k; si++) s += b->T[(size_t)ri * b->k + si] * vc[b->S[si]];
        vc[b->R[ri]] -= s;
      }
      /* L: v_J -= E v_R */
      for (int a = 0; a < b->nj; a++) {
        double s = 0.0;
        for (int ri = 0; ri < b->r; ri++) s += b->E[(size_t)a * b->r + ri] * vc[b->R[ri]];
        vc[b->J[a]] -= s;
      }
    }
    for (int i = 0; i < F->nbox; i++) {
      obox *b = &F->box[i];
      double *xi = malloc(sizeof(double) * (b->r + 1));
      for (int ri = 0; ri < b->r; ri++) xi[ri] = vc[b->R[ri]];
      lu_solve(b->LU, b->piv, b->r, xi, 1);
      for (int ri = 0; ri < b->r; ri++) vc[b->R[ri]] = xi[ri];
      free(xi);
    }
    int nt = F->ntop;
    double *xt = malloc(sizeof(double) * (nt + 1));
    for (int i = 0; i < nt; i++) xt[i] = vc[F->top[i]];
    lu_solve(F->LUtop, F->pivtop, nt, xt, 1);
    for (int i = 0; i < nt; i++) vc[F->top[i]] = xt[i];
    free(xt);
    for (int i = F->nbox - 1; i >= 0; i--) {
      obox *b = &F->box[i];
      /* U: v_R -= G v_J */
      for (int ri = 0; ri < b->r; ri++) {
        double s = 0.0;
        for (int a = 0; a < b->nj; a++) s += b->G[(size_t)ri * b->nj + a] * vc[b->J[a]];
        vc[b->R[ri]] -= s;
      }
      /* L_T: v_S -= T v_R */
      for (int si = 0; si < b->k; si++) {
        double s = 0.0;
        for (int ri = 0; ri < b->r; ri++) s += b->T[(size_t)ri * b->k + si] * vc[b->R[ri]];
        vc[b->S[si]] -= s;
      }
    }
  }
  from_tree(F, v, x, nrhs);
  free(v);
}

/* Generalized square root (the remark after Eq. 3.11): for positive definite
 * K the factors are symmetric (V_i = W_i^T), and with D = L L^T by
 * Cholesky blocks, F^{1/2} = (prod V_i) P_t L satisfies F = F^{1/2}
 * (F^{1/2})^T.  X_RR of each box is rebuilt from its stored LU and pivots
 * (row piv[i] of X_RR is row i of L U), then factored by Cholesky; the top
 * block likewise.  Returns 0, or 1 + the index of the first block that is
 * not positive definite (the factors are then left unset). */
static int chol_from_lu(const double *LU, const int *piv, int r, double *C) {
  double *X = malloc(sizeof(double) * ((size_t)r * r + 1));
  for (int i = 0; i < r; i++)
    for (int j = 0; j < r; j++) {
      double s = 0.0;
      for (int l = 0; l <= (i < j ? i : j); l++) s += (l == i ? 1.0 : LU[(size_t)i * r + l]) * LU[(size_t)l * r + j];
      X[(size_t)piv[i] * r + j] = s;
    }
  /* lower Cholesky factor, row-major, of the symmetric part */
  int ok = 1;
  for (int j = 0; j < r && ok; j++) {
    double d = 0.5 * (X[(size_t)j * r + j] + X[(size_t)j * r + j]);
    for (int l = 0; l < j; l++) d -= C[(size_t)j * r + l] * C[(size_t)j * r + l];
    if (!(d > 0.0)) {
      ok = 0;
      break;
    }
    C[(size_t)j * r + j] = sqrt(d);
    for (int i = j + 1; i < r; i++) {
      double s = 0.5 * (X[(size_t)i * r + j] + X[(size_t)j * r + i]);
      for (int l = 0; l < j; l++) s -= C[(size_t)i * r + l] * C[(size_t)j * r + l];
      C[(size_t)i * r + j] = s / C[(size_t)j * r + j];
    }
    for (int i = 0; i < j; i++) C[(size_t)i * r + j] = 0.0;
  }
  free(X);
  return ok;
}

int orc_sqrt_prepare(void *h) {
  ofactor *F = h;
  if (F->chol) return 0;
  double **C = calloc((size_t)F->nbox + 1, sizeof(double *));
  for (int i = 0; i <= F->nbox; i++) {
    int r = i < F->nbox ? F->box[i].r : F->ntop;
    const double *LU = i < F->nbox ? F->box[i].LU : F->LUtop;
    const int *piv = i < F->nbox ? F->box[i].piv : F->pivtop;
    C[i] = calloc((size_t)r * r + 1, sizeof(double));
    if (!chol_from_lu(LU, piv, r, C[i])) {
      for (int q = 0; q <= i; q++) free(C[q]);
      free(C);
      return i + 1;
    }
  }
  F->chol = C;
  return 0;
}

/* y = F^{1/2} x (trans = 0) or (F^{1/2})^T x (trans = 1); orc_sqrt_prepare
 * first.  x, y: n x nrhs column-major in the caller's point order. */
void orc_sqrt_apply(void *h, const double *x, double *y, int nrhs, int trans) {
  ofactor *F = h;
  int64_t n = F->T->n;
  double *v = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * nrhs);
  to_tree(F, x, v, nrhs);
  for (int c = 0; c < nrhs; c++) {
    double *vc = v + (size_t)c * n;
    if (trans) { /* the W product, as in orc_apply */
      for (int i = 0; i < F->nbox; i++) {
        obox *b = &F->box[i];
        for (int si = 0; si < b->k; si++) {
          double s = 0.0;
          for (int ri = 0; ri < b->r; ri++) s += b->T[(size_t)ri * b->k + si] * vc[b->R[ri]];
          vc[b->S[si]] += s;
        }
        for (int ri = 0; ri < b->r; ri++) {
          double s = 0.0;
          for (int a = 0; a < b->nj; a++) s += b->G[(size_t)ri * b->nj + a] * vc[b->J[a]];
          vc[b->R[ri]] += s;
        }
      }
    }
    /* the Cholesky blocks: L (trans = 0) or L^T (trans = 1) */
    for (int i = 0; i <= F->nbox; i++) {
      int r = i < F->nbox ? F->box[i].r : F->ntop;
      const int64_t *ids = i < F->nbox ? F->box[i].R : F->top;
      const double *L = F->chol[i];
      double *t = malloc(sizeof(double) * (r + 1));
      for (int a = 0; a < r; a++) {
        double s = 0.0;
        for (int l = 0; l < r; l++) s += (trans ? L[(size_t)l * r + a] : L[(size_t)a * r + l]) * vc[ids[l]];
        t[a] = s;
      }
      for (int a = 0; a < r; a++) vc[ids[a]] = t[a];
      free(t);
    }
    if (!trans) { /* the V product, as in orc_apply */
      for (int i = F->nbox - 1; i >= 0; i--) {
        obox *b = &F->box[i];
        for (int a = 0; a < b->nj; a++) {
          double s = 0.0;
          for (int ri = 0; ri < b->r; ri++) s += b->E[(size_t)a * b->r + ri] * vc[b->R[ri]];
          vc[b->J[a]] += s;
        }
        for (int ri = 0; ri < b->r; ri++) {
          double s = 0.0;
          for (int si = 0; si < b->k; si++) s += b->T[(size_t)ri * b->k + si] * vc[b->S[si]];
          vc[b->R[ri]] += s;
        }
      }
    }
  }
  from_tree(F, v, y, nrhs);
  free(v);
}

/* ------------------------------------------------------------------------ */
/* Exact references                                                           */
/* ------------------------------------------------------------------------ */

/* Dense A (n x n row-major) in the caller's point order. */
void orc_dense_matrix(const double *pts, int64_t n, int dim, int kind, double diag, double w,
                      double *A) {
  okern kn = {kind, dim, diag, w};
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = 0; j < n; j++) A[i * n + j] = entry(&kn, pts, i, j);
}

/* y = A x by direct summation, rows `rows` only (all rows if rows == NULL,
 * nrows = n).  x: n x nrhs col-major; y: nrows x nrhs col-major. */
void orc_matvec_rows(const double *pts, int64_t n, int dim, int kind, double diag, double w,
                     const double *x, int nrhs, const int64_t *rows, int64_t nrows, double *y) {
  okern kn = {kind, dim, diag, w};
  for (int64_t q = 0; q < nrows; q++) {
    int64_t i = rows ? rows[q] : q;
    for (int c = 0; c < nrhs; c++) {
      double s = 0.0;
      for (int64_t j = 0; j < n; j++) s += entry(&kn, pts, i, j) * x[(size_t)c * n + j];
      y[(size_t)c * nrows + q] = s;
    }
  }
}

/* Worst ratio residual / bound over all boxes (check mode): what 0 the CPQR
 * ID bound, 1 proxy validity. */
double orc_factor_check_worst(void *h, int what) {
  ofactor *F = h;
  return what == 0 ? F->id_worst : F->proxy_worst;
}

/* Solve A X = B with a plain right-looking LU with partial pivoting.
 * A n x n row-major (overwritten), B n x nrhs col-major (overwritten with X).
 * Returns the LU info code. */
int orc_dense_solve(double *A, int n, double *B, int nrhs) {
  int *piv = malloc(sizeof(int) * (n + 1));
  int info = orc_lu(A, n, piv);
  if (!info) lu_solve(A, piv, n, B, nrhs);
  free(piv);
  return info;
}
