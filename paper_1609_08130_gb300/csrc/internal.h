// internal.h -- structures shared by the host orchestration (api.cu) and the
// device kernels (kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rss {

// One strongly skeletonized box: where its part of the factor lives.
// Sizes k, r, nj are written by the device kernels; capacities by the host.
template <typename T> struct FBox {
  int cell;   // cell id within its level
  int depth;  // tree depth t of the box
  int b;      // |B| (active DOFs at the start of the level)
  int k, r;   // |S|, |R| (device-written)
  int nj;     // |J| = k + |N| (device-written)
  int njmax;  // capacity bound on nj
  int no;     // |O| active DOFs in the ring inside the proxy surface (device-written)
  int rres;   // |R| and |J| the storage below was reserved for (LU, Xi: rres^2;
  int njres;  // E, G: njres * rres each); a box that does not fit takes overflow space
  int64_t *ids; // [b] global tree-order ids: S (pivot order) then R
  int *loc;     // [b] local indices in the cell's level layout, same order
  int64_t *J;   // [njmax] global ids of J = [S; N]
  int *Jnb;     // [njmax] 3^d-neighbourhood code of each J entry's cell
  int *Jloc;    // [njmax] local index of each J entry in its cell
  T *Tm;        // k x r column-major (ld k): T = R11^{-1} R12
  T *LU;        // r x r row-major, L\U of P X_RR
  int *piv;     // [r] row i of P X_RR is row piv[i] of X_RR
  T *Xi;        // r x r column-major: X_RR^{-1} = U^{-1} L^{-1} P formed from the LU
  T *E;         // nj x r column-major (ld nj): E = X_JR X_RR^{-1}
  T *G;         // r x nj column-major (ld r):  G = X_RR^{-1} X_RJ
};

// Overflow space of one level: a box whose rank left r > rres takes
// 2 r^2 + 2 njmax r elements here (bump allocation); when it is exhausted the
// box records DERR_CAPACITY and the factorization is redone with full-size
// reservations.
template <typename T> struct Overflow {
  T *base;
  unsigned long long *used;  // elements taken so far
  int64_t cap;               // elements available (0: none)
};

// Device view of one level (depth t): the cells holding active DOFs, their
// neighbour tables and the pool of pair blocks at Chebyshev distance <= 2.
// Pair block (c, o) holds rows = cell c's level-start DOFs, columns = the
// level-start DOFs of neighbour nbr[c*NB+o], column-major with ld = b_c.
template <typename T> struct LevelDev {
  int t, dim, ncell, NB;
  const int *cell_b;
  const int64_t *cell_dof_off;  // [ncell+1]
  const int64_t *cell_dofs;     // tree-order ids, ascending within a cell
  const int *cell_coord;        // [3*ncell]
  const int *cell_nbr;          // [ncell*NB] or -1
  const int64_t *pair_off;      // [ncell*NB] element offset into pool or -1
  int *act_cnt;                 // [ncell] active count
  int *act_idx;                 // [sum b] active local indices, ascending
  const int *dof_cell;          // [n] cell of each active DOF at this level
  const int *dof_loc;           // [n] local index of each active DOF
  T *pool;
  int shared;                   // 1: boxes of one phase may share pair blocks
                                // (2^d colours): Schur updates add atomically
  int weak;                     // 1: weak skeletonization (RS-WS, Sec. 3.4):
                                // the ID compresses against every cell inside
                                // the proxy surface, J = S
};

// A list of dense blocks to assemble: block q has rows row_ids[row_off[q] ..
// + nrow[q]) and columns col_ids[col_off[q] .. + ncol[q]), written
// column-major (ld nrow[q]) at out + out_off[q] (or its transpose).  Entries whose two DOFs sat
// at Chebyshev distance <= 2 in the previous level are copied from that
// level's pool (they may carry Schur-complement updates); all others are
// kernel entries (Corollary 3.2: unmodified far-field interactions).
struct AssembleList {
  int nblock;
  const int64_t *row_off, *col_off, *out_off;
  const int *nrow, *ncol;
  const int64_t *row_ids, *col_ids;
  int transpose;  // 1: entry (i, j) holds A(col j, row i) (row-major A)
  // level mode (cell_nbr set): block q is the pair (cell q / NB, neighbour
  // code q % NB), read from the level's tables; row_off .. ncol are unused
  const int *cell_nbr, *cell_b;
  const int64_t *cell_dof_off, *pair_off;
  int NB;
};

struct ProxyParams {
  int np;
  double radius;
};

// Launchers (kernels.cu).  All run on `st`.
template <typename T>
void launch_assemble(const AssembleList &L, T *out, const LevelDev<T> *prev, const Points &P,
                     const KernelParams &K, int64_t maxblk, cudaStream_t st);
template <typename T>
void launch_id(const LevelDev<T> &lv, FBox<T> *boxes, const int *box_list, int nbox, int bmax,
               int mmax, const Points &P, const KernelParams &K, const ProxyParams &px,
               const T *proxy_unit, double eps, T *gscratch, int64_t gscratch_stride, bool use_smem,
               cudaStream_t st, int *err);
// Launch shape of the next ID launch on this thread: CTAs per box << 8 |
// threads per column << 4 | fold groups per box (0: default).
void set_id_groups(int G);
// Shape of the next elimination launch of this thread (k_elim2 path):
// (split << 4) | CTAs per box, 0 for the built-in choice.
void set_elim_shape(int h);
// Scratch of the multi-CTA ID: triangle slots (slot_elems elements each,
// max_slots of them; none for boxes wider than 512) and tree-node counters
// (8 x max_slots ints, zero between launches).  kid_ctas: CTAs per box of
// the general kernel k_id (its workspaces are the level's ID scratch, which
// then holds kid_ctas of them per box).
struct IdMultiScratch {
  void *tri = nullptr;
  int64_t slot_elems = 0, max_slots = 0;
  int *cnt = nullptr;
  int kid_ctas = 0;
};
void set_id_multi(const IdMultiScratch &m);
template <typename T>
void launch_elim(const LevelDev<T> &lv, FBox<T> *boxes, const int *box_list, int nbox, int bmax,
                 T *scratch, int64_t scratch_stride, const Overflow<T> &ovf, cudaStream_t st, int *err, int njmax);
template <typename T>
void launch_schur(const LevelDev<T> &lv, const FBox<T> *boxes, const int *box_list, int nbox,
                  int njmax, const T *scratch, int64_t scratch_stride, cudaStream_t st);
// The FP32 factor's Schur update on the tensor cores (schur_tc.cu): the same
// arguments as launch_schur plus the device error word (a bounded wait that
// gives up records DERR_INTERNAL).
void launch_schur_tc(const LevelDev<float> &lv, const FBox<float> *boxes, const int *box_list, int nbox, int njmax,
                     const float *scratch, int64_t scratch_stride, cudaStream_t st, int *err);
template <typename T>
void launch_dense_lu(T *A, int n, int *piv, T *W, cudaStream_t st, int *err);
// Per-box sums of log|U_jj| (part[0..nbox), and a DOF id of each box in
// first[]) and per-problem sums over the top blocks' LU (part[nbox..)).
template <typename T>
void launch_logdet(const FBox<T> *boxes, int nbox, const T *topLU, const int64_t *loff, const int *tn, int nprob,
                   double *part, int64_t *first, cudaStream_t st);

// Sweeps over the factor (kernels.cu).  v: tree-order working vector,
// layout v[g * nrhs + c].
// shared != 0: boxes of the phase may share near DOFs (2^d colours), whose
// updates are then atomic additions.
template <typename T>
void launch_sweep(int mode, const FBox<T> *boxes, int first, int count, T *v, int nrhs, int bmax,
                  int njmax, cudaStream_t st, int shared = 0);
// Solve sweeps over work items (box, chunk of SWEEP_CHUNK rows of J) for
// nrhs <= 4; cnt: per-box counters (zero between launches); pbuf/poff: the
// backward sweep's per-box partial sums (ceil(nj / SWEEP_CHUNK) x r x 4
// elements per box).  Shared memory as sweep_chunk_smem.
constexpr int SWEEP_CHUNK = 128;
template <typename T>
void launch_sweep_chunks(int mode, const FBox<T> *boxes, const int *wbox, const int *wchunk, int nwork, T *v,
                         int nrhs, int bmax, int *cnt, T *pbuf, const int64_t *poff, cudaStream_t st,
                         int shared = 0);
size_t sweep_chunk_smem(int bmax, int nrhs, int elem);
// Set the shared-memory attributes of every sweep kernel on the current device.
void sweep_kernel_attributes();
// Top blocks: mode 0 solves with the LU factors (or, for one problem with
// Winv = U^{-1} L^{-1} and at most 4 columns, multiplies by it), mode 1
// multiplies by the block.  launch_top_inverse forms Winv (n <= 1024).
template <typename T>
void launch_top(int mode, const T *LU, const int64_t *loff, const int *piv, const int64_t *top, const int64_t *toff,
                const int *tn, int nprob, int ntop_total, T *v, int nrhs, T *work, cudaStream_t st,
                const T *Winv = nullptr);
template <typename T> void launch_top_inverse(const T *LU, int n, T *W, cudaStream_t st);
template <typename T>
void launch_lu_batched(T *LU, const int64_t *loff, int *piv, const int64_t *toff, const int *tn, int nprob,
                       cudaStream_t st, int *err);
// Per level: act_idx[j] = local index of level DOF j in its cell; for each
// level DOF g: dof_cell[g] = its cell, dof_loc[g] = its local index.
void launch_level_maps(int ncell, const int64_t *cell_dof_off, const int64_t *cell_dofs, int *act_idx, int *dof_cell,
                       int *dof_loc, cudaStream_t st);
template <typename T> int64_t id_region_bytes(int b, int PR);
template <typename T> int64_t elim_ws_elems(int bmax);
template <typename T>
void launch_permute(int dir, const int64_t *perm, const double *in, T *out_or_in, double *out,
                    int64_t n, int nrhs, cudaStream_t st);
void launch_matvec(const double *x_tree, int dim, const KernelParams &K, const double *wdof, const int64_t *perm,
                   const double *xin, double *yout, int64_t n, int nrhs, int ntile, const int64_t *tstart,
                   const int64_t *tend, const int64_t *sbeg, const int64_t *send, cudaStream_t st);
// The same product with the kernel evaluated and summed in FP32 (the
// points' distances from their depth-20 cells and offsets, as the FP32
// factor's blocks; each tile of 256 sources summed in FP32, the tiles in
// FP64): the operator of the inner GMRES of the refinement.
void launch_matvec_f32(const Points &P, const KernelParams &K, const int64_t *perm, const double *xin,
                       double *yout, int64_t n, int nrhs, int ntile, const int64_t *tstart, const int64_t *tend,
                       const int64_t *sbeg, const int64_t *send, cudaStream_t st);

// FP64 operator x -> A x for points on an s^d grid of cell centres, by FFT
// convolution on the circulant of side L = 2s (refine.cu).
struct GridOp {
  int dim = 0, s = 0, L = 0, logL = 0;
  int64_t n = 0;
  double h = 0, w = 0, diag = 1;
  int kind = 0;
  const int64_t *gidx = nullptr;  // grid linear index of each point (caller order)
  double2 *C = nullptr;           // spectrum of the embedded kernel
  double2 *X = nullptr;           // work
  double2 *tw = nullptr;          // twiddles
  float2 *Cf = nullptr, *Xf = nullptr, *twf = nullptr;  // the same in FP32 (inner products of GMRES-IR)
};
void grid_op_setup(GridOp &G, cudaStream_t st);
// Cf and twf rounded from C and tw (after grid_op_setup; Cf, Xf, twf allocated by the caller)
void grid_op_setup_f32(GridOp &G, cudaStream_t st);
// y = A x for nrhs columns; f32: the transforms in FP32 (y still FP64)
void grid_op_apply(const GridOp &G, const double *x, double *y, int nrhs, cudaStream_t st, bool f32);
void multidot(const double *V, int64_t vstride, int nv, const double *w, int64_t n, int nrhs, double *part,
              double *out, cudaStream_t st);
void combine(double *y, double alpha, const double *V, int64_t vstride, int nv, const double *coef, int64_t n,
             int nrhs, cudaStream_t st);

// Rank-proposal network (mlp.cu).  Features per box: MLP_NFEAT FP32 values;
// parameters: MLP_NPARAM (layout in mlp.cu); wbf: their bfloat16 copy.
constexpr int MLP_NFEAT = 16, MLP_HIDDEN = 64;
constexpr int MLP_NPARAM = MLP_HIDDEN * MLP_NFEAT + MLP_HIDDEN + 2 * (MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN) +
                           MLP_HIDDEN + 1;
void mlp_round(const float *theta, void *wbf, cudaStream_t st);
void mlp_forward(const void *wbf, const float *X, int64_t n, float *out, cudaStream_t st);
int mlp_grad_blocks(int64_t n);
void mlp_gradient(const void *wbf, const float *X, const float *y, int64_t n, float *part, double *lpart, float *grad,
                  double *loss, cudaStream_t st);
void mlp_adam(float *theta, float *m, float *v, const float *grad, void *wbf, int *step, float lr,
              cudaStream_t st);

// The adaptive tree on the GPU (tree.cu).  Points of nprob problems,
// concatenated (problem p's first point is pofs[p], device array of nprob + 1);
// prob_bits: bits for the problem index above the 20 dim Morton key bits
// (dim * 20 + prob_bits <= 64).  tree_gpu_sort sorts and counts the nodes
// (total at T.total, device); tree_gpu_nodes writes the nodes in pre-order
// (start: sorted position) and the tree-order permutation, coordinates,
// depth-20 cells and Morton keys.
struct TreeGpu {
  const double *pts = nullptr;
  int64_t n = 0;
  int dim = 2, leaf = 64;
  const int64_t *pofs = nullptr;
  int nprob = 1, prob_bits = 0;
  uint64_t *k0 = nullptr, *k1 = nullptr, *mkey = nullptr;
  int64_t *i0 = nullptr, *i1 = nullptr;
  int *c20 = nullptr, *c20s = nullptr, *Lp = nullptr;
  uint32_t *nd = nullptr, *hist = nullptr, *total = nullptr;
  int64_t nblk = 0;
};
int64_t tree_gpu_scratch_bytes(int64_t n, int dim);
void tree_gpu_sort(TreeGpu &T, void *scratch, cudaStream_t st);
void tree_gpu_nodes(const TreeGpu &T, int *depth, int *parent, int *coord, int64_t *start, int64_t *count,
                    int64_t *perm, double *x, int *c20t, uint64_t *keyt, cudaStream_t st);
// A factor's per-point arrays (cells padded to 3 coordinates, FP32 offsets
// from the cell corners) and the grid test of the FFT residual operator,
// both from the tree-order points on the device.
void points_setup(const double *x, const int *c20, int64_t n, int dim, double D, int *cell3, float *off,
                  cudaStream_t st);
void grid_detect(const double *x, const int64_t *perm, int64_t n, int dim, int64_t s, int64_t *gidx, unsigned *seen,
                 int *bad, cudaStream_t st);

// A level's lists for one problem on the GPU (tree.cu).  level_gpu_keys:
// the depth-t keys of the active DOFs (act, na of them, ascending tree
// order; ksh = dim (20 - t)), *unsorted set when they are not in key order
// (the caller then sorts keys and DOFs stably); level_gpu_runs: run starts
// of the key-ordered list, their exclusive scan and the cell count at
// *ncell.  level_gpu_tables (ncell known): the cells' DOF lists,
// sizes, keys and coordinates, the neighbour table and pair-block offsets
// (5^dim codes per cell; the pool size at *pool_total, the largest cell at
// *bmax), and per tree node of depth t (node_coord, 3 ints each) six ints:
// cell (-1: no active DOF), b, DOFs of the cell and its near cells, DOFs of
// its ring cells, near and ring cells present.  level_gpu_next_active: the active DOFs after the
// level's eliminations (act_cnt / act_idx per cell), their number at *total.
struct LevelGpu {
  const int64_t *act = nullptr;
  int64_t na = 0;
  int dim = 2, NB = 25, side = 1, ncell = 0, nbox = 0;
  const uint64_t *dk = nullptr;
  const uint32_t *flag = nullptr, *cpos = nullptr;
  const int *node_coord = nullptr;
  int *grid = nullptr;  // side^dim cells, or nullptr for binary search
  int64_t *cell_dof_off = nullptr, *cell_dofs = nullptr, *pair_off = nullptr;
  int *cell_b = nullptr, *cell_coord = nullptr, *cell_nbr = nullptr, *bmax = nullptr, *box_out = nullptr;
  uint64_t *cell_key = nullptr;
  unsigned long long *psz = nullptr, *pool_total = nullptr;
};
void level_gpu_keys(const uint64_t *key, const int64_t *act, int64_t na, int ksh, uint64_t *dk, uint32_t *unsorted,
                    cudaStream_t st);
void level_gpu_runs(const uint64_t *dk, int64_t na, uint32_t *flag, uint32_t *cpos, uint32_t *ncell, cudaStream_t st);
// Stable LSD radix sort of n (key, value) pairs by the low `bits` bits of
// the keys, 8 bits a pass; the result is in (k0, v0); k1, v1 and hist
// (sort_pairs_hist_bytes(n)) are scratch.
int64_t sort_pairs_hist_bytes(int64_t n);
void sort_pairs_u64(uint64_t *k0, int64_t *v0, uint64_t *k1, int64_t *v1, uint32_t *hist, int64_t n, int bits,
                    cudaStream_t st);
void level_gpu_tables(const LevelGpu &L, cudaStream_t st);
void level_gpu_next_active(int ncell, const int64_t *cell_dof_off, const int64_t *cell_dofs, const int *act_cnt,
                           const int *act_idx, uint32_t *aoff, uint32_t *total, int64_t *next, cudaStream_t st);
void iota64(int64_t *p, int64_t n, cudaStream_t st);  // p[i] = i

// Process-wide count of kernel launches made by this library.
void count_launch(int n = 1);
long long launches_total();

// Sweep modes.  SWEEP_APPLY_W: the forward apply sweep without the
// diagonal block (the W product of the generalized square root).
enum { SWEEP_SOLVE_FWD = 0, SWEEP_SOLVE_BWD = 1, SWEEP_APPLY_FWD = 2, SWEEP_APPLY_BWD = 3, SWEEP_APPLY_W = 4 };

// Generalized square root: lower Cholesky factors of the boxes' X_RR and the
// problems' top blocks (block q at C + coff[q], boxes first), rebuilt from
// their LU factors; and v_B := C v_B or C^T v_B on every block's DOFs
// (rmax: the largest block order).
template <typename T>
void launch_chol_from_lu(const FBox<T> *boxes, int nbox, const T *topLU, const int64_t *loff, const int *toppiv,
                         const int64_t *toff, const int *tn, int nprob, T *C, const int64_t *coff, int *err,
                         cudaStream_t st);
template <typename T>
void launch_chol_apply(const FBox<T> *boxes, int nbox, const int64_t *top, const int64_t *toff, const int *tn,
                       int nprob, const T *C, const int64_t *coff, T *v, int nrhs, int rmax, int trans,
                       cudaStream_t st);

}  // namespace rss
