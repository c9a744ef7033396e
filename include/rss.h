/*
 * rss.h -- C ABI of the GB300 implementation of the strong recursive
 * skeletonization factorization (RS-S) of Minden, Ho, Damle & Ying,
 * "A recursive skeletonization factorization based on strong admissibility"
 * (arXiv:1609.08130).
 *
 * The matrix factored is the second-kind discretisation
 *     A = diag * I + w * K,   K_ij = K(x_i - x_j) (i != j),  K_ii = 0,
 * of the integral equation of Sec. 1 (Eq. 1.1, 1.3), with the 2D Laplace
 * kernel K(z) = -log|z| / (2 pi) (Sec. 3.2, Example 1) or the 3D Laplace
 * kernel K(z) = 1 / (4 pi |z|) (Example 2).
 *
 * Conventions shared by every entry point:
 *   - Points are DEVICE memory, FP64, point-major (x0 y0 [z0] x1 y1 ...).
 *   - Vectors are DEVICE memory, FP64, in the caller's original point order;
 *     several right-hand sides are column-major (n x nrhs, leading dim n).
 *   - The caller owns every buffer it passes; the library owns handles until
 *     rss_free.  No pointer passed in is kept after the call returns, except
 *     that a factor keeps its own copy of the points.
 *   - Calls run on the stream given in rss_options (NULL: the legacy default
 *     stream) and return after their work is complete (they synchronise the
 *     stream), so outputs may be read on return -- unless the factor was
 *     made with RSS_FLAG_ASYNC (see there).
 *   - Errors are reported by the return code; rss_last_error() gives a
 *     thread-local message.  No C++ exception crosses the ABI.
 */
#ifndef RSS_H
#define RSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RSS_OK = 0,
  RSS_EINVAL = 1,   /* bad argument (sizes, pointers, kind, eps, leaf) */
  RSS_ENOMEM = 2,   /* device or host allocation failed */
  RSS_ECUDA = 3,    /* a CUDA runtime call failed */
  RSS_ENUMERIC = 4, /* an exactly singular pivot block was met */
  RSS_ETIMEOUT = 5, /* a bounded device wait gave up (not used by this path) */
  RSS_ENOTCONV = 6  /* iterative refinement did not reach the tolerance */
} rss_status;

typedef enum { RSS_LAPLACE2D_LOG = 0, RSS_LAPLACE3D_INV = 1 } rss_kernel_kind;

/* Matrix A = diag * I + weight * K; weight <= 0 selects 1/N. */
typedef struct {
  int kind;      /* rss_kernel_kind */
  double diag;   /* 1.0 for the second-kind problems */
  double weight; /* quadrature weight w; <= 0 means 1/N */
} rss_kernel;

typedef enum { RSS_FP64 = 0, RSS_MIXED = 1 } rss_precision;

typedef struct rss_mlp rss_mlp; /* rank-proposal network (rss_mlp_create) */

typedef struct {
  int prec;            /* rss_precision: FP64 everywhere, or an FP32 factor */
  int n_proxy;         /* proxy points; 0: 64 (2D) / 512 (3D) (Sec. 4) */
  double proxy_radius; /* in box sides; 0: 2.5 (Sec. 3.2) */
  int use_graphs;      /* 1: each solve with nrhs <= 4 replays a CUDA graph
                          of its launch sequence, captured on first use */
  void *stream;        /* cudaStream_t; NULL = legacy default stream */
  int profile;         /* 1: time every kernel launch with CUDA events on the
                          stream (see rss_profile) */
  int flags;           /* RSS_FLAG_* bits; 0 for the defaults */
  const rss_mlp *mlp;  /* rank proposal presizing the factor storage, or NULL
                          (see rss_mlp_create); borrowed for the call only */
} rss_options;

/* Route every box through the plain one-CTA-per-box kernels with
 * global-memory workspaces (the general ID and elimination), which otherwise
 * run only for boxes too wide for the other forms, and then over several
 * CTAs per box.  The result is the same factorization up to rounding; the
 * tests compare the other paths with it. */
#define RSS_FLAG_LARGE_BOX_PATH 1
/* Use the built-in launch shapes instead of the autotuner's choices (see
 * rss_autotune_table). */
#define RSS_FLAG_NO_AUTOTUNE 2
/* The paper's parallel schedule with 2^dim colours per level (Sec. 5: boxes
 * of one colour are two or more cells apart) instead of the default 3^dim
 * colours.  Boxes of one colour phase are skeletonized at once from the
 * state at the phase start: each one's ID sees the other boxes of the phase
 * still whole in its ring, and two boxes may share near-field blocks, whose
 * Schur-complement updates (and the solve's and apply's updates of shared
 * near-field entries) are added atomically.  The result is a different but
 * equally valid factorization, with 2^dim instead of 3^dim phases per level;
 * the order of the atomic additions makes it reproducible only up to
 * rounding.  rss_tree_query keeps reporting the 3^dim order. */
#define RSS_FLAG_COLOUR_2D 4
/* Run the FP32 factor's Schur-complement updates on the FP32 SIMT units
 * instead of the tensor cores (which use a three-product TF32 split that
 * keeps FP32 accuracy); the same factorization up to rounding.  For
 * comparisons; the FP64 factor always uses FP64 SIMT arithmetic. */
#define RSS_FLAG_NO_TENSOR_CORES 8
/* Symmetric storage: both kernels are symmetric, so G = X_RR^{-1} X_RJ is
 * E^T (E = X_JR X_RR^{-1}; Sec. 3.3, V_i = W_i^T) and only E is kept: the
 * boxes' factor storage drops by |J| r entries each (the largest share),
 * and the sweeps read E transposed where they read G.  The same
 * factorization up to rounding. */
#define RSS_FLAG_SYMMETRIC_STORAGE 16
/* The hybrid factorization RS-WS (Sec. 3.4, Algorithm 2) instead of RS-S: at
 * every depth each box is first weakly skeletonized -- its ID compresses its
 * interactions with every cell inside the proxy surface and, through the
 * proxy points, the rest, and its redundant DOFs are eliminated against its
 * skeleton alone (J = S) -- then what stays active is strongly
 * skeletonized as in RS-S; a last weak pass runs at depth 1.  Fewer stored
 * entries and a smaller top block, at a somewhat larger apply error.  Not
 * with RSS_FLAG_COLOUR_2D or a rank proposal (RSS_EINVAL). */
#define RSS_FLAG_HYBRID 32
/* Asynchronous calls.  rss_factor returns once the last level's ranks are
 * known and the top block's LU is queued; rss_apply, rss_solve,
 * rss_solve_noalloc, rss_sqrt_apply (after its first call) and rss_matvec
 * return once their work is queued on the stream.  Their outputs may be
 * read after the stream has been synchronised (by the caller, or by
 * rss_sync).  An error the device records in that work (a zero pivot in the
 * top block) is returned by the next call on the factor that finds the work
 * finished, and at the latest by rss_sync.  rss_solve_refined,
 * rss_solve_cg and rss_logdet stay synchronous (they read device results
 * on the host).  Ignored when profiling (options.profile), which reads
 * CUDA events after every call. */
#define RSS_FLAG_ASYNC 64

typedef struct rss_tree rss_tree;
typedef struct rss_factorization rss_factorization;

/* rss_build_tree -- adaptive quadtree (dim 2) / octree (dim 3) on [0,1]^dim,
 * nodes split while they hold more than leaf_size points (Sec. 3: "each leaf
 * box contains a bounded number of DOFs"; Sec. 4: refine until n_occ per
 * leaf), at most depth 20.  Integer cell of coordinate v at depth t is
 * floor(v 2^t) clamped to [0, 2^t - 1]; child index = sum_d bit_d << d; the
 * DOF order is the stable pre-order of the tree (children ascending, points
 * of a leaf in original order).
 *   pts: device, n*dim doubles.  n >= 0; dim in {2,3}; leaf_size >= 1.
 *   out: receives a handle owned by the caller (free with rss_free).
 * Errors: RSS_EINVAL on bad sizes / NULL out; RSS_ECUDA, RSS_ENOMEM. */
rss_status rss_build_tree(const double *pts, int64_t n, int dim, int leaf_size, rss_tree **out);

/* rss_tree_query -- copy a tree array into a HOST buffer.
 * what:  0 perm (int64[n], original index of tree-order DOF g)
 *        1 node depth (int32[nnode])   2 node parent (int32[nnode], -1 root)
 *        3 node coords (int32[3*nnode]) 4 node start (int64[nnode])
 *        5 node count (int64[nnode])   6 sizes (int64[4]: nnode, maxdepth, n, dim)
 *        100+t  boxes of depth t in elimination order (int32[]): colour-major
 *               with 3^dim colours c = sum_d (coord_d mod 3) 3^d, Morton order
 *               within a colour (the paper's order is "fixed but arbitrary",
 *               Sec. 3.3.1; same-colour boxes are >= 3 apart, Sec. 5)
 *        200+t  per box of depth t (same order): neighbour cells holding
 *               points at depth t, int32 records {nnear, nring, codes...}
 *               with codes sum_d (delta_d + 2) 5^d ascending, near first.
 * buf may be NULL to ask for the size; *nbytes is in/out (capacity/size).
 * Errors: RSS_EINVAL for an unknown `what` or a too-small buffer (the size
 * needed is still written to *nbytes). */
rss_status rss_tree_query(const rss_tree *tree, int what, void *buf, size_t *nbytes);

/* rss_factor -- RS-S factorization F ~ A (Algorithm 1, Eq. 3.10).  Boxes of
 * depths maxdepth..2 are strongly skeletonized level by level (Sec. 3.3):
 * an ID of the box's interactions with the ring of boxes inside the proxy
 * surface and with the proxy points (Eq. 3.7) splits it into skeleton and
 * redundant DOFs, then the redundant DOFs are eliminated against the
 * skeleton and near field (Eq. 3.4).  The remaining DOFs form the top block,
 * factored by LU.
 *   pts: device, n*dim doubles (a private copy is kept).
 *   eps: ID tolerance, >= 0 (0 keeps every column: F = A up to rounding).
 *   leaf_size: as in rss_build_tree.  opts: may be NULL (defaults).
 * Errors: RSS_EINVAL, RSS_ENOMEM, RSS_ECUDA, RSS_ENUMERIC (zero pivot). */
rss_status rss_factor(const double *pts, int64_t n, int dim, rss_kernel kernel, double eps,
                      int leaf_size, const rss_options *opts, rss_factorization **out);

/* rss_factor_batched -- factor nprob independent problems into one handle
 * (the matrix is block diagonal, one block per problem; problem p's weight is
 * kernel.weight or 1/n[p]).  Every (tree depth, colour) phase is one launch
 * over the boxes of all problems (the boxes of one colour are independent
 * within a problem and across problems).
 *   pts: HOST array of nprob DEVICE pointers (n[p]*dim doubles each);
 *   n: HOST array of nprob sizes.  Vectors passed to rss_apply / rss_solve /
 *   rss_solve_refined on the handle are the problems' vectors concatenated in
 *   problem order (sum n[p] rows).  Errors as rss_factor. */
rss_status rss_factor_batched(int nprob, const double *const *pts, const int64_t *n, int dim, rss_kernel kernel,
                              double eps, int leaf_size, const rss_options *opts, rss_factorization **out);

/* rss_apply -- y = F x (Eq. 3.10).  x, y: device, n x nrhs column-major,
 * original point order; may not alias.  nrhs >= 1. */
rss_status rss_apply(const rss_factorization *f, const double *x, double *y, int nrhs);

/* rss_solve -- x = F^{-1} b (Eq. 3.11).  b, x: device, n x nrhs column-major;
 * may not alias.  nrhs >= 1. */
rss_status rss_solve(const rss_factorization *f, const double *b, double *x, int nrhs);

/* rss_solve_noalloc -- x = F^{-1} b, the same result as rss_solve, for callers
 * that must not have the library allocate device memory during the call:
 * programs that hand all device memory to their own allocator up front, or
 * that keep a fixed memory budget inside a hot loop and cannot afford an
 * allocation's cost or failure there.  rss_solve may allocate a working
 * vector on its first use with a given number of right-hand sides; this
 * variant never does.  The paper has no counterpart to this entry point.
 *   Working space is one fixed 16 MiB array in device memory that exists
 *   once per device from the moment the library is loaded until the process
 *   exits.  The columns are solved in passes (as rss_solve does, at most as
 *   many columns as the sweep kernels' shared memory takes, and fewer if the
 *   array needs it); a pass of c columns keeps n x c plus 2 * ntop * c
 *   entries there, in the factor's precision (4 bytes for a RSS_MIXED
 *   factor, 8 for RSS_FP64).  If a single column does not fit (about 4.19 M
 *   points for RSS_MIXED, 2.09 M for RSS_FP64, less twice the top-block
 *   size), the call returns RSS_EINVAL without doing any work.  Nothing in
 *   the array needs to start at zero: every pass overwrites what it reads.
 *   The first call made with a given device current looks up the array's
 *   device address (cudaGetSymbolAddress) and raises the sweep kernels'
 *   shared-memory limits on that device; make that first call before any
 *   stream capture begins.
 *   Every call uses the same array: calls whose work overlaps on the GPU
 *   (different streams, different host threads) race and give wrong
 *   results.  Calls serialised on one stream are safe.
 *   b, x: device, n x nrhs column-major, may not alias; the caller owns
 *   them.  nrhs >= 1.  Errors: RSS_EINVAL, RSS_ECUDA. */
rss_status rss_solve_noalloc(const rss_factorization *f, const double *b, double *x, int nrhs);

/* rss_solve_refined -- solve A x = b to a relative residual
 * max_c ||b_c - A x_c|| / ||b_c|| <= tol by GMRES-based iterative refinement
 * (Carson & Higham): x0 = F^{-1} b, then FP64 residuals with the exact
 * operator (rss_matvec) and corrections from restarted FGMRES(10) in FP64,
 * right-preconditioned by the factor's solve (which runs in FP32 for a
 * RSS_MIXED factor; for such a factor FGMRES's operator products are FP32
 * too, on FP64 vectors, while the residuals and the update stay FP64).  The paper uses F as a CG preconditioner instead
 * (Sec. 4); GMRES is used here because a FP32 factor is not symmetric to
 * FP64 accuracy.
 *   b, x: device, n x nrhs column-major, may not alias.  maxit: outer
 *   refinement steps (>= 0).  iters (may be NULL): total inner iterations;
 *   relres (may be NULL): final relative residual (max over columns).
 * Errors: RSS_EINVAL; RSS_ENOTCONV when tol is not met within maxit
 * (x then holds the last iterate). */
rss_status rss_solve_refined(const rss_factorization *f, const double *b, double *x, int nrhs, double tol,
                             int maxit, int *iters, double *relres);

/* rss_solve_cg -- solve A x = b to a relative residual
 * max_c ||b_c - A x_c|| / ||b_c|| <= tol by conjugate gradients
 * preconditioned with the factor, the paper's iterative solver for its
 * examples (Sec. 4; A and F are symmetric for these kernels, V_i = W_i^T):
 * x0 = F^{-1} b, FP64 vectors and residuals with the exact operator
 * (rss_matvec), z = F^{-1} r as preconditioner (FP32 for a RSS_MIXED factor;
 * beta in the flexible Polak-Ribiere form, which tolerates the FP32 factor's
 * small asymmetry).  The true residual is checked when the recurrence
 * residual meets tol, and CG restarts from x if it does not.
 *   b, x: device, n x nrhs column-major, may not alias.  maxit: iterations
 *   (>= 0).  iters (may be NULL): iterations taken; relres (may be NULL):
 *   final true relative residual (max over columns).
 * Errors: RSS_EINVAL; RSS_ENOTCONV when tol is not met within maxit
 * (x then holds the last iterate). */
rss_status rss_solve_cg(const rss_factorization *f, const double *b, double *x, int nrhs, double tol, int maxit,
                        int *iters, double *relres);

/* rss_sqrt_apply -- y = F^{1/2} x (transpose = 0) or y = (F^{1/2})^T x
 * (transpose = 1), the generalized square root of the remark after
 * Eq. 3.11: for symmetric positive definite A the factor is F = V D V^T
 * (W = V^T), and with D = C C^T (C the block lower triangular Cholesky
 * factors of every box's X_RR and of the top blocks) F^{1/2} = V C, so that
 * F = F^{1/2} (F^{1/2})^T.  The Cholesky factors are rebuilt from the stored
 * LU factors on the first call (X = P^T L U, then the factor of its
 * symmetric part) and kept with the factorization.  x, y: device, n x nrhs
 * column-major, may not alias.  Errors: RSS_EINVAL (bad arguments, a top
 * block larger than 4096); RSS_ENUMERIC when a diagonal block is not
 * positive definite (A is not). */
rss_status rss_sqrt_apply(const rss_factorization *f, const double *x, double *y, int nrhs, int transpose);

/* rss_matvec -- y = A x in FP64 with the exact operator being factored:
 * an FFT convolution when the points are the cell centres of an s^dim grid
 * (s a power of two; exact up to FP64 rounding), direct summation over all
 * pairs otherwise (the 2D kernel's logarithm table-driven, to a few units
 * of FP64 rounding).  Device buffers, n x nrhs column-major. */
rss_status rss_matvec(const rss_factorization *f, const double *x, double *y, int nrhs);

/* rss_sync -- wait for the factor's stream, then report an error the device
 * recorded in work of an asynchronous call (RSS_FLAG_ASYNC) that no call has
 * reported yet (RSS_ENUMERIC for a zero pivot in the top block); RSS_OK
 * otherwise.  Each recorded error is reported once. */
rss_status rss_sync(const rss_factorization *f);

/* rss_logdet -- log |det F| of the factorization F ~ A (Sec. 3.3, the
 * determinant by-product: the factors U_T, L_T and the elimination's unit
 * triangular factors have determinant 1, so det F is the product of the
 * determinants of every box's X_RR and of the top block).  Computed as the
 * sum of log |U_jj| over the LU factors the factorization stores, in
 * double.  logabs: HOST array, one entry per problem (1 for rss_factor,
 * nprob for rss_factor_batched).  Synchronous.  RSS_EINVAL for a NULL
 * argument. */
rss_status rss_logdet(const rss_factorization *f, double *logabs);

/* rss_stats -- factor statistics into a HOST int64 array:
 *   [0] number of skeletonized boxes  [1] top-block size  [2] factor bytes
 *   [3] maxdepth                      [4] n               [5] precision
 *   [6] bytes reserved for the boxes' T, LU, X_RR^{-1}, E and G (with the
 *       overflow space when a rank proposal was used)
 *   [7] bytes those arrays need at the ranks found: sum of k r + 2 r^2 + 2 nj r
 *   [8] overflow bytes taken by boxes whose r exceeded their reservation
 *   [9] 1 when a proposal left a level short and the factorization was redone
 *       with full-size reservations, else 0
 *  [10] 1 when the reservations came from a rank proposal (options.mlp)
 * followed, per box in elimination order, by {depth, b, k, nj, rres, njres}
 * (rres, njres: the r and |J| its storage was reserved for).  *nbytes in/out
 * as in rss_tree_query. */
rss_status rss_stats(const rss_factorization *f, int64_t *buf, size_t *nbytes);

/* rss_stats_json -- the factor's statistics as a NUL-terminated JSON
 * document in a HOST buffer: sizes (n, problems, dim, precision, eps, colour
 * phases per level, maxdepth, boxes, top-block size), storage (factor,
 * reserved, used and overflow bytes; whether a rank proposal was used and
 * whether the factorization was redone), per depth the boxes and the sums
 * and maxima of |B|, k and |J| (the skeleton ranks of Sec. 3.3), per box in
 * elimination order its depth, |B|, k and |J|, and the kernel-class times
 * in milliseconds when the factor was created with options.profile.
 * buf may be NULL to ask for the size; *nbytes in/out as in
 * rss_tree_query (the size includes the terminating NUL). */
rss_status rss_stats_json(const rss_factorization *f, char *buf, size_t *nbytes);

/* rss_profile -- per-kernel-class totals of a factor created with
 * options.profile = 1, accumulated over rss_factor and every later
 * rss_apply / rss_solve on it, into a HOST double array of 4 * 13 entries:
 * for class c in {0 assemble, 1 id, 2 elim, 3 schur, 4 top LU, 5 sweep,
 * 6 top solve/multiply, 7 permute, 8 host tree build, 9 host level build,
 * 10 host wait at level end, 11 FP64 residual operator, 12 FP32 operator
 * products inside the refinement's GMRES}: {launches or calls,
 * milliseconds (CUDA events on the launching stream; host wall time for the
 * host classes), algorithmic bytes, algorithmic flops}.  The algorithmic
 * counts are the data the method must move or compute (stated per class in
 * the implementation), not hardware counters.
 * reset != 0 clears the totals after copying.  *nbytes in/out. */
rss_status rss_profile(const rss_factorization *f, int reset, double *buf, size_t *nbytes);

/* Rank proposal (not in the paper).  A small network predicts each box's
 * skeleton fraction k/b from features known before its ID; rss_factor with
 * options.mlp reserves each box's LU, X_RR^{-1}, E and G for the predicted
 * r = b - k and |J| = k + (near DOFs still active at the box's turn: the
 * predicted skeletons of neighbours eliminated in an earlier colour phase,
 * all DOFs of the others), each plus a margin, instead of for r = b and the
 * level-start |J|.  The column-pivoted QR still
 * decides every rank (Sec. 2.2, Definition 2.1): a box that does not fit its
 * reservation takes the level's overflow space, and if that runs out the
 * factorization is redone with full-size reservations (rss_stats [9]).  The
 * factor is the same either way.
 *
 * Network: 16 features -> 64 -> 64 -> 64 (tanh) -> 1, parameters one FP32
 * vector of RSS_MLP_NPARAM values in the order W1 (64 x 16 row-major, row =
 * output unit), b1, W2 (64 x 64), b2, W3 (64 x 64), b3, w4 (64), b4.  The
 * forward and backward passes read the parameters rounded to bfloat16 and
 * compute in FP32; Adam keeps the FP32 master copy.  Features per box (FP32):
 *   0 dim == 3    1 kernel kind    2 -log10(eps)/10    3 log2(1+b)/10
 *   4 log2(1+|N|)/10 (near DOFs)   5 log2(1+|O|)/10 (ring DOFs, Sec. 3.2)
 *   6 near cells present/(3^d-1)   7 ring cells present/(5^d-3^d)
 *   8 leaf box    9 b / (sum of the children's b), 1 for a leaf
 *  10 depth/10   11 log2(1+n_p)/10  12 proxy radius/5   13..15 zero. */
#define RSS_MLP_NFEAT 16
#define RSS_MLP_NPARAM 9473

/* rss_mlp_create -- a network on `stream` (cudaStream_t, NULL = legacy
 * default).  params: HOST array of RSS_MLP_NPARAM FP32 values, or NULL for
 * Glorot-uniform weights from SplitMix64(seed) (uniform = top 53 bits of
 * output i times 2^-53 for flat parameter i) and zero biases.  Free with
 * rss_free.  Errors: RSS_EINVAL, RSS_ENOMEM, RSS_ECUDA. */
rss_status rss_mlp_create(const float *params, uint64_t seed, void *stream, rss_mlp **out);

/* rss_mlp_params -- copy the FP32 master parameters to a HOST array of
 * RSS_MLP_NPARAM values. */
rss_status rss_mlp_params(const rss_mlp *m, float *params);

/* rss_mlp_predict -- y[i] = network(X[i]) for n samples.  X: DEVICE, n x 16
 * FP32 row-major; y: DEVICE, n FP32. */
rss_status rss_mlp_predict(const rss_mlp *m, const float *X, int64_t n, float *y);

/* rss_mlp_grad -- gradient of the loss mean_i (network(X[i]) - y[i])^2 with
 * respect to the parameters (DEVICE, RSS_MLP_NPARAM FP32, same order), and the
 * loss (HOST double, may be NULL).  X, y: DEVICE, n >= 1 samples. */
rss_status rss_mlp_grad(const rss_mlp *m, const float *X, const float *y, int64_t n, float *grad, double *loss);

/* rss_mlp_train -- `iters` full-batch Adam steps (beta1 0.9, beta2 0.999,
 * eps 1e-8, learning rate lr) on the loss above; the step counter persists
 * across calls.  *loss (HOST, may be NULL): the loss before the last step. */
rss_status rss_mlp_train(rss_mlp *m, const float *X, const float *y, int64_t n, int iters, float lr,
                         double *loss);

/* rss_box_features -- every skeletonized box's features (HOST, nbox x 16
 * FP32, elimination order as in rss_stats) and the rank k its ID found (HOST,
 * nbox int32): training data for the network.  nbox must equal rss_stats [0]. */
rss_status rss_box_features(const rss_factorization *f, float *feat, int32_t *rank, int64_t nbox);

/* rss_autotune_table -- the autotuner's choices so far in this process, as
 * HOST int32 records of 25: {element bytes (4 FP32 factor, 8 FP64), box-width
 * class (64, 128 or 256), phase-size class (floor(log2(boxes in the phase))),
 * the chosen shape (threads per column, fold groups per box, CTAs per box,
 * panel rows per thread in units of 32 FP32 / 16 FP64 rows), then the
 * measured time in microseconds of the 18 candidate shapes = (1,1,1,1)
 * (1,2,1,1) (1,4,1,1) (2,1,1,1) (2,2,1,1) (2,4,1,1) (4,1,1,1) (4,2,1,1)
 * (2,1,4,1) (2,1,8,1) (4,1,4,1) (4,1,8,1) (0,2,1,1) (0,4,1,1) (0,8,1,1)
 * (1,1,1,2) (1,2,1,2) (1,4,1,2) (0: not a candidate)}.
 * The ID kernel (Sec. 2.2: Householder reduction of the ID matrix to a
 * triangle, then greedy column pivoting) splits each column over threads
 * that keep 32 (FP32) or 16 (FP64) rows of every panel (twice that with two
 * units of rows), a box's rows over fold groups of one CTA or over several
 * CTAs, whose triangles are merged by a tree; more threads per box mean
 * fewer sequential steps per box, fewer fit more boxes per SM.  Threads per
 * column 0 (width class 64 only) is the warp-per-panel form: `groups`
 * warps per box, each folding its own panels with the box's columns spread
 * over its 32 lanes, two per lane, the panels pipelined into one triangle.  The first colour phase that meets a key times
 * every candidate on its own boxes (the ID launch is idempotent), keeps the
 * fastest for the rest of the process and re-runs it, so factorizations
 * with the same key compute the same result.  Disabled per factorization by
 * RSS_FLAG_NO_AUTOTUNE.  *nbytes in/out as in rss_tree_query. */
rss_status rss_autotune_table(int32_t *buf, size_t *nbytes);

/* rss_autotune_set -- fix the shape used for one key (e.g. a table saved
 * from another run), without timing.  Errors: RSS_EINVAL for a shape that is
 * not a candidate or exceeds the kernel's thread limit (256 threads for one
 * thread per column, 512 otherwise; the 256 width class takes several CTAs
 * per box only with two threads per column; the warp-per-panel form only
 * the 64 width class; two units of rows only one thread per column and
 * width classes 64 and 128). */
rss_status rss_autotune_set(int elem_bytes, int width, int phase_class, int tpc, int groups, int ctas, int rows);

/* rss_autotune_elim_table -- the elimination's autotuned shapes so far in
 * this process, as HOST int32 records of 10: {element bytes, box-width class
 * (64 or 128), phase-size class, chosen split flag and CTAs per box, then the
 * measured time in microseconds of the 5 candidates (split, CTAs per box) =
 * (0,1) (1,1) (1,2) (1,4) (1,8)}.  Split 0 forms E and G in the same kernel
 * as the LU of X_RR, one CTA per box; split 1 leaves X_JR and X_RJ in scratch
 * for a phase-wide product kernel, the box's rows of J shared by that many
 * CTAs.  The first phase of a key times every candidate (the elimination of
 * a phase writes the same values however often it runs), keeps the fastest
 * and re-runs it.  Not tuned with a rank proposal, on the large-box path, or
 * with RSS_FLAG_NO_AUTOTUNE.  *nbytes in/out as in rss_tree_query. */
rss_status rss_autotune_elim_table(int32_t *buf, size_t *nbytes);

/* rss_autotune_clear -- forget every choice (ID and elimination); the next
 * factorizations tune again. */
void rss_autotune_clear(void);

/* rss_free -- release a tree, factor or network handle (NULL-safe). */
void rss_free(void *handle);

/* rss_kernel_launches -- number of CUDA kernel launches this library has
 * made in this process (all devices, all handles). */
int64_t rss_kernel_launches(void);

/* rss_last_error -- message of the last failing call on this thread. */
const char *rss_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RSS_H */
