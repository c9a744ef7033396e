// kernels.cu -- CUDA kernels (sm_103a) for the strong recursive
// skeletonization factorization (RS-S) and its apply / solve sweeps.
//
// Per level (tree depth t) and per colour phase, every box of the phase is
// skeletonized independently (same-colour boxes are >= 3 cells apart, so
// their 3^d neighbourhoods -- everything a box reads or writes -- are
// disjoint):
//   k_id     : ID of the box (Definition 2.1) from the rows of its
//              interactions with the ring O inside the proxy surface and the
//              proxy rows (Eq. 3.7), by a shared-memory Householder
//              reduction of those rows to a b x b triangle followed by
//              greedy column-pivoted QR of the triangle;
//   k_elim   : the operators U_T, L_T (Sec. 3.1) and the elimination of the
//              redundant DOFs: LU of X_RR, E = X_JR X_RR^{-1},
//              G = X_RR^{-1} X_RJ (Sec. 2.1, Eq. 3.4);
//   k_schur  : X_JJ -= E G scattered into the pair blocks of the level.
// k_assemble builds the pair blocks of a level (Corollary 3.2: entries not
// reached by any Schur update are kernel entries) and the top block.
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "internal.h"

namespace rss {

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

constexpr int NT = 256;  // threads per CTA for the per-box kernels
constexpr int SWEEP_TROWS = 4;  // rows of T^T v_S a warp of the forward sweep forms at once
constexpr int SWEEP_MLP = 8;    // independent loads a sweep thread keeps in flight

// Kernel attributes are set outside stream capture only (a captured launch
// reuses the attribute set by an earlier uncaptured one).
static bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// ---------------------------------------------------------------------------
// Assembly of pair blocks / top block
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(NT) k_assemble(AssembleList L, T *__restrict__ out, LevelDev<T> prev,
                                                 int has_prev, Points P, KernelParams K) {
  const int q = blockIdx.x;
  int nr, nc;
  const int64_t *rid, *cid;
  T *o;
  if (L.cell_nbr) {
    const int nb = L.cell_nbr[q];
    if (nb < 0) return;
    const int c = q / L.NB;
    nr = L.cell_b[c];
    nc = L.cell_b[nb];
    rid = L.row_ids + L.cell_dof_off[c];
    cid = L.col_ids + L.cell_dof_off[nb];
    o = out + L.pair_off[q];
  } else {
    nr = L.nrow[q];
    nc = L.ncol[q];
    rid = L.row_ids + L.row_off[q];
    cid = L.col_ids + L.col_off[q];
    o = out + L.out_off[q];
  }
  const int64_t tot = (int64_t)nr * nc;
  // element e = (i, j) of the column-major block: e / nr by a multiply-high
  // while the block has fewer than 2^31 entries (every pair block; the top
  // block up to 46340 DOFs)
  const bool small = tot < ((int64_t)1 << 31);
  const FastDiv fnr(max(nr, 1));
  const T wT = (T)K.w, dT = (T)K.diag;  // converted once per CTA, not once per entry
  for (int64_t e = blockIdx.y * (int64_t)NT + threadIdx.x; e < tot; e += (int64_t)NT * gridDim.y) {
    int i, j;
    if (small) {
      fnr.divmod((int)e, j, i);
    } else {
      i = (int)(e % nr);
      j = (int)(e / nr);
    }
    int64_t gi = rid[i], gj = cid[j];
    if (L.transpose) {
      int64_t tg = gi;
      gi = gj;
      gj = tg;
    }
    T v;
    bool done = false;
    // A DOF without a cell at the previous level belongs to a problem whose
    // tree is shallower than the merged previous level: none of its entries
    // has been updated yet, so the kernel entry is the value.
    int ci = has_prev ? prev.dof_cell[gi] : -1, cj = has_prev ? prev.dof_cell[gj] : -1;
    if (ci >= 0 && cj >= 0) {
      int dx = prev.cell_coord[3 * cj] - prev.cell_coord[3 * ci];
      int dy = prev.cell_coord[3 * cj + 1] - prev.cell_coord[3 * ci + 1];
      int dz = prev.cell_coord[3 * cj + 2] - prev.cell_coord[3 * ci + 2];
      if (dx >= -2 && dx <= 2 && dy >= -2 && dy <= 2 && dz >= -2 && dz <= 2) {
        int64_t off = prev.pair_off[(int64_t)ci * prev.NB + code5(dx, dy, dz, prev.dim)];
        v = prev.pool[off + prev.dof_loc[gi] + (int64_t)prev.dof_loc[gj] * prev.cell_b[ci]];
        done = true;
      }
    }
    if (!done) v = P.wdof ? entry<T>(P, K, gi, gj) : entry_t<T>(P, K.kind, wT, dT, gi, gj);
    o[e] = v;
  }
}

// The same for the pair blocks of a level whose cells hold at most AS_MAX
// DOFs (level mode, no per-DOF weights): one CTA per block, the block's row
// and column DOFs staged first -- their points, and their previous-level
// cell, its coordinates and the DOF's place in it -- so that each entry is
// a copy from the previous level's pool or a kernel evaluation from shared
// memory.
constexpr int AS_MAX = 128;
template <typename T> struct AsPts;
template <> struct AsPts<float> {
  int c[3][AS_MAX];
  float o[3][AS_MAX];
};
template <> struct AsPts<double> {
  double x[3][AS_MAX];
};
struct AsPrev {
  int cell[AS_MAX], loc[AS_MAX], cc[3][AS_MAX];
};

template <typename T>
__global__ void __launch_bounds__(NT) k_assemble_staged(AssembleList L, T *__restrict__ out, LevelDev<T> prev,
                                                        int has_prev, Points P, KernelParams K) {
  __shared__ AsPts<T> sp[2];  // rows, columns
  __shared__ AsPrev spv[2];
  const int q = blockIdx.x;
  const int nb = L.cell_nbr[q];
  if (nb < 0) return;
  const int c = q / L.NB;
  const int nr = L.cell_b[c], nc = L.cell_b[nb];
  const int64_t *ids[2] = {L.row_ids + L.cell_dof_off[c], L.col_ids + L.cell_dof_off[nb]};
  const int cnt[2] = {nr, nc};
  T *o = out + L.pair_off[q];
  const int dim = P.dim;
  for (int s = 0; s < 2; s++)
    for (int i = threadIdx.x; i < cnt[s]; i += NT) {
      const int64_t g = ids[s][i];
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
          sp[s].c[d][i] = P.cell[3 * g + d];
          sp[s].o[d][i] = P.off[3 * g + d];
        }
      } else {
#pragma unroll
        for (int d = 0; d < 3; d++) sp[s].x[d][i] = d < dim ? P.x[g * dim + d] : 0.0;
      }
      const int pc = has_prev ? prev.dof_cell[g] : -1;
      spv[s].cell[i] = pc;
      spv[s].loc[i] = pc >= 0 ? prev.dof_loc[g] : 0;
#pragma unroll
      for (int d = 0; d < 3; d++) spv[s].cc[d][i] = pc >= 0 ? prev.cell_coord[3 * pc + d] : 0;
    }
  __syncthreads();
  const T wT = (T)K.w, dT = (T)K.diag;
  const FastDiv fnr(max(nr, 1));
  for (int e = threadIdx.x; e < nr * nc; e += NT) {
    int i, j;
    fnr.divmod(e, j, i);
    T v;
    bool done = false;
    const int ci = spv[0].cell[i], cj = spv[1].cell[j];
    if (ci >= 0 && cj >= 0) {
      const int dx = spv[1].cc[0][j] - spv[0].cc[0][i], dy = spv[1].cc[1][j] - spv[0].cc[1][i],
                dz = spv[1].cc[2][j] - spv[0].cc[2][i];
      if (dx >= -2 && dx <= 2 && dy >= -2 && dy <= 2 && dz >= -2 && dz <= 2) {
        const int64_t off = prev.pair_off[(int64_t)ci * prev.NB + code5(dx, dy, dz, prev.dim)];
        v = prev.pool[off + spv[0].loc[i] + (int64_t)spv[1].loc[j] * prev.cell_b[ci]];
        done = true;
      }
    }
    if (!done) {
      if (ids[0][i] == ids[1][j]) {
        v = dT;
      } else {
        T r2;
        if constexpr (sizeof(T) == 4) {
          const float Dd = P.D;
          const float ex = fmaf((float)(sp[0].c[0][i] - sp[1].c[0][j]), Dd, sp[0].o[0][i] - sp[1].o[0][j]);
          const float ey = fmaf((float)(sp[0].c[1][i] - sp[1].c[1][j]), Dd, sp[0].o[1][i] - sp[1].o[1][j]);
          r2 = ex * ex + ey * ey;
          if (dim == 3) {
            const float ez = fmaf((float)(sp[0].c[2][i] - sp[1].c[2][j]), Dd, sp[0].o[2][i] - sp[1].o[2][j]);
            r2 = fmaf(ez, ez, r2);
          }
        } else {
          const double ex = sp[0].x[0][i] - sp[1].x[0][j], ey = sp[0].x[1][i] - sp[1].x[1][j];
          r2 = ex * ex + ey * ey;
          if (dim == 3) {
            const double ez = sp[0].x[2][i] - sp[1].x[2][j];
            r2 += ez * ez;
          }
        }
        v = wT * kof(K.kind, r2);
      }
    }
    o[e] = v;
  }
}

template <typename T>
void launch_assemble(const AssembleList &L, T *out, const LevelDev<T> *prev, const Points &P,
                     const KernelParams &K, int64_t maxblk, cudaStream_t st) {
  if (L.nblock == 0) return;
  LevelDev<T> pv{};
  if (prev) pv = *prev;
  if (L.cell_nbr && !P.wdof && maxblk <= (int64_t)AS_MAX * AS_MAX) {
    k_assemble_staged<T><<<L.nblock, NT, 0, st>>>(L, out, pv, prev ? 1 : 0, P, K);
    count_launch();
    return;
  }
  int gy = (int)((maxblk + NT * 8 - 1) / (NT * 8));
  if (gy < 1) gy = 1;
  if (gy > 1024) gy = 1024;
  dim3 grid(L.nblock, gy);
  k_assemble<T><<<grid, NT, 0, st>>>(L, out, pv, prev ? 1 : 0, P, K); count_launch();
}

// One warp per cell: local indices of its level DOFs and the per-DOF maps.
__global__ void k_level_maps(int ncell, const int64_t *__restrict__ off, const int64_t *__restrict__ dofs,
                             int *act_idx, int *dof_cell, int *dof_loc) {
  const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (c >= ncell) return;
  const int64_t o = off[c], e = off[c + 1];
  for (int64_t j = o + lane; j < e; j += 32) {
    const int q = (int)(j - o);
    const int64_t g = dofs[j];
    act_idx[j] = q;
    dof_cell[g] = c;
    dof_loc[g] = q;
  }
}

void launch_level_maps(int ncell, const int64_t *cell_dof_off, const int64_t *cell_dofs, int *act_idx, int *dof_cell,
                       int *dof_loc, cudaStream_t st) {
  if (ncell <= 0) return;
  const int64_t threads = (int64_t)ncell * 32;
  k_level_maps<<<(unsigned)((threads + NT - 1) / NT), NT, 0, st>>>(ncell, cell_dof_off, cell_dofs, act_idx, dof_cell,
                                                                 dof_loc);
  count_launch();
}

// ---------------------------------------------------------------------------
// ID: Householder reduction of the proxy-compressed far-field rows, then
// greedy column-pivoted QR of the b x b triangle.
// ---------------------------------------------------------------------------

template <typename T> struct IdLayout {
  // offsets in elements of T within the per-box region
  int ldr, ldp;
  int64_t oR, oP, oN, oPerm;  // oPerm in elements of T (ints placed after)
  int64_t bytes;
  __host__ __device__ IdLayout(int b, int PR) {
    ldr = b + 1;
    ldp = PR + 1;
    oR = 0;
    oP = oR + (int64_t)ldr * b;
    oN = oP + (int64_t)ldp * b;
    oPerm = oN + b;
    bytes = oPerm * (int64_t)sizeof(T) + (int64_t)b * sizeof(int) + 16;
  }
};

template <typename T>
__global__ void __launch_bounds__(NT) k_id(LevelDev<T> lv, FBox<T> *boxes, const int *box_list, Points P,
                                           KernelParams K, ProxyParams px, double eps, int PR, T *gscr,
                                           int64_t gstride, int use_smem, int C, int *cnt, int *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ocell[125], s_obase[126], s_ono;
  __shared__ int64_t s_rowsrc[256];
  __shared__ T s_r11, s_hh[3];
  __shared__ int s_stop, s_piv, s_k, s_second;

  // C CTAs per box (global workspaces only): CTA `chunk` folds panels
  // chunk, chunk + C, ... of the ID matrix into the triangle of its own
  // workspace; the triangles are merged up a binary tree (at each node the
  // second CTA to arrive, told by a counter, folds the right triangle into
  // the left one) and the CTA left at the root pivots.
  const int bq = blockIdx.x / C, chunk = blockIdx.x % C;
  FBox<T> &fb = boxes[box_list[bq]];
  const int c = fb.cell, b = fb.b, dim = lv.dim;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = NT / 32;
  IdLayout<T> lay(b, PR);
  T *base = use_smem ? reinterpret_cast<T *>(smem_raw) : gscr + (int64_t)blockIdx.x * gstride;
  T *R = base + lay.oR;
  // the panel: in this CTA's workspace, or with several CTAs per box in
  // shared memory (PR x b, the launch sizes PR to fit)
  T *pan = C > 1 ? reinterpret_cast<T *>(smem_raw) : base + lay.oP;
  T *nrm = base + lay.oN;
  int *perm = reinterpret_cast<int *>(base + lay.oPerm);
  const int ldr = lay.ldr, ldp = lay.ldp;

  for (int e = tid; e < ldr * b; e += NT) R[e] = (T)0;
  // Ring O: cells at Chebyshev distance exactly 2 with active DOFs.
  if (tid == 0) {
    int no = 0, acc = 0;
    int lim = dim == 3 ? 2 : 0;
    for (int dz = -lim; dz <= lim; dz++)
      for (int dy = -2; dy <= 2; dy++)
        for (int dx = -2; dx <= 2; dx++) {
          int m = max(abs(dx), max(abs(dy), abs(dz)));
          if (m != 2 && !(lv.weak && m == 1)) continue;  // ring O; weak steps: N too
          int code = code5(dx, dy, dz, dim);
          int nb = lv.cell_nbr[(int64_t)c * lv.NB + code];
          if (nb < 0) continue;
          int cnt = lv.act_cnt[nb];
          if (cnt <= 0) continue;
          s_ocell[no] = code;  // store the code; the cell is looked up again
          s_obase[no] = acc;
          acc += cnt;
          no++;
        }
    s_obase[no] = acc;
    s_ono = no;
  }
  __syncthreads();
  const int no = s_ono;
  const int nO = s_obase[no];
  const int m = nO + px.np;
  const int64_t coff = lv.cell_dof_off[c];
  const T w = (T)weight_of(P, K, lv.cell_dofs[lv.cell_dof_off[c]]);
  // proxy circle / sphere about the box centre (Sec. 3.2)
  const double D = ldexp(1.0, -lv.t);
  double ctr[3];
  for (int d = 0; d < 3; d++) ctr[d] = (lv.cell_coord[3 * c + d] + 0.5) * D;

  // [R; panel] -> R, one Householder reflector per column from column j0 on
  // (the panel's entries left of j0 are zero).  Several CTAs per box: warp 0
  // forms reflector j, then each thread updates its columns of the panel
  // (shared memory, lanes on consecutive columns) and of row j of R.  One
  // CTA per box: each warp updates its columns with warp-wide dot products.
  auto fold_panel = [&](int rows, int j0) {
    if (C > 1) {
      for (int j = j0; j < b; j++) {
        const T *pj = pan + (int64_t)j * ldp;
        if (warp == 0) {
          T s = (T)0;
          for (int i = lane; i < rows; i += 32) s += pj[i] * pj[i];
          s = warp_sum(s);
          if (lane == 0) {
            if (s > (T)0) {
              const T x0 = R[j + (int64_t)j * ldr];
              const T nrm2 = sqrt(x0 * x0 + s);
              const T beta = x0 >= (T)0 ? -nrm2 : nrm2;
              s_hh[0] = (beta - x0) / beta;
              s_hh[1] = (T)1 / (x0 - beta);
              s_hh[2] = (T)1;
              R[j + (int64_t)j * ldr] = beta;  // no other thread reads R_jj
            } else {
              s_hh[2] = (T)0;
            }
          }
        }
        __syncthreads();
        if (s_hh[2] != (T)0) {
          const T tau = s_hh[0], scl = s_hh[1];
          for (int cc = j + 1 + tid; cc < b; cc += NT) {
            T *pc = pan + (int64_t)cc * ldp;
            const T rj = R[j + (int64_t)cc * ldr];
            T d0 = (T)0, d1 = (T)0, d2 = (T)0, d3 = (T)0;
            int i = 0;
            for (; i + 3 < rows; i += 4) {
              d0 += pj[i] * pc[i];
              d1 += pj[i + 1] * pc[i + 1];
              d2 += pj[i + 2] * pc[i + 2];
              d3 += pj[i + 3] * pc[i + 3];
            }
            for (; i < rows; i++) d0 += pj[i] * pc[i];
            const T f = tau * (rj + scl * ((d0 + d1) + (d2 + d3)));
            const T fs = f * scl;
            for (i = 0; i < rows; i++) pc[i] -= fs * pj[i];
            R[j + (int64_t)cc * ldr] = rj - f;
          }
        }
        __syncthreads();
      }
      return;
    }
    for (int j = j0; j < b; j++) {
      const T *pj = pan + (int64_t)j * ldp;
      T s = (T)0;
      for (int i = lane; i < rows; i += 32) s += pj[i] * pj[i];
      s = warp_sum(s);
      if (s > (T)0) {
        T x0 = R[j + (int64_t)j * ldr];
        T nrm2 = sqrt(x0 * x0 + s);
        T beta = x0 >= (T)0 ? -nrm2 : nrm2;
        T tau = (beta - x0) / beta;
        T scl = (T)1 / (x0 - beta);
        for (int cc = j + 1 + warp; cc < b; cc += nwarp) {
          T *pc = pan + (int64_t)cc * ldp;
          T d = (T)0;
          for (int i = lane; i < rows; i += 32) d += pj[i] * pc[i];
          d = warp_sum(d);
          T wv = R[j + (int64_t)cc * ldr] + scl * d;
          T f = tau * wv;
          T fs = f * scl;
          for (int i = lane; i < rows; i += 32) pc[i] -= fs * pj[i];
          if (lane == 0) R[j + (int64_t)cc * ldr] -= f;
        }
      }
      __syncthreads();
      // every warp has read x0 = R_jj; now it may be replaced by beta
      if (s > (T)0 && tid == 0) {
        T x0 = R[j + (int64_t)j * ldr];
        T nrm2 = sqrt(x0 * x0 + s);
        R[j + (int64_t)j * ldr] = x0 >= (T)0 ? -nrm2 : nrm2;
      }
    }
    __syncthreads();
  };
  for (int p0 = chunk * PR; p0 < m; p0 += C * PR) {
    const int rows = min(PR, m - p0);
    // row sources of this panel
    for (int rr = tid; rr < rows; rr += NT) {
      int row = p0 + rr;
      int64_t src;
      if (row < nO) {
        int q = 0;
        while (s_obase[q + 1] <= row) q++;
        int code = s_ocell[q];
        int nb = lv.cell_nbr[(int64_t)c * lv.NB + code];
        int loc = lv.act_idx[lv.cell_dof_off[nb] + (row - s_obase[q])];
        // column `loc` of pair block (c, nb): rows are the box's DOFs
        src = lv.pair_off[(int64_t)c * lv.NB + code] + (int64_t)loc * b;
      } else {
        src = -1 - (int64_t)(row - nO);
      }
      s_rowsrc[rr] = src;
    }
    __syncthreads();
    for (int e = tid; e < rows * b; e += NT) {
      int rr = e / b, q = e % b;
      int64_t src = s_rowsrc[rr];
      T v;
      if (src >= 0) {
        v = lv.pool[src + q];
      } else {
        int mm = (int)(-1 - src);
        double y[3];
        if (dim == 2) {
          double th = 2.0 * kPi * (double)mm / (double)px.np;
          y[0] = ctr[0] + px.radius * D * cos(th);
          y[1] = ctr[1] + px.radius * D * sin(th);
          y[2] = 0.0;
        } else {
          double z = 1.0 - (2.0 * mm + 1.0) / (double)px.np;
          double rr2 = sqrt(1.0 - z * z);
          double ph = (double)mm * kPi * (3.0 - sqrt(5.0));
          y[0] = ctr[0] + px.radius * D * rr2 * cos(ph);
          y[1] = ctr[1] + px.radius * D * rr2 * sin(ph);
          y[2] = ctr[2] + px.radius * D * z;
        }
        int64_t g = lv.cell_dofs[coff + q];
        const double *xg = P.x + g * dim;
        double r2 = 0.0;
        for (int d = 0; d < dim; d++) {
          double dd = y[d] - xg[d];
          r2 += dd * dd;
        }
        v = w * kof(K.kind, (T)r2);
      }
      pan[rr + (int64_t)q * ldp] = v;
    }
    for (int e = tid; e < (PR - rows) * b; e += NT) {
      int rr = rows + e / b, q = e % b;
      pan[rr + (int64_t)q * ldp] = (T)0;
    }
    __syncthreads();
    fold_panel(rows, 0);
  }
  int cur = chunk;  // first workspace of the subtree this CTA carries
  for (int L = 1; L < C; L <<= 1) {
    const int ls = cur & ~(2 * L - 1), rs = ls + L;
    if (rs >= C) continue;  // no right partner at this level: carry the subtree up
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      int *node = cnt + ((int64_t)bq * 8 + (31 - __clz(L))) * C + ls;
      const int seen = atomicAdd(node, 1);
      s_second = seen == 1;
      if (seen == 1) *node = 0;  // reset for the next launch
    }
    __syncthreads();
    if (!s_second) return;
    __threadfence();
    if (cur != ls) R = gscr + ((int64_t)bq * C + ls) * gstride + lay.oR;  // continue on the left triangle
    const T *Rr = gscr + ((int64_t)bq * C + rs) * gstride + lay.oR;
    for (int p0 = 0; p0 < b; p0 += PR) {  // rows p0.. of the right triangle are zero left of column p0
      const int rows = min(PR, b - p0);
      for (int e = tid; e < PR * b; e += NT) {
        const int rr = e % PR, q = e / PR;
        pan[rr + (int64_t)q * ldp] = rr < rows ? __ldcg(Rr + (p0 + rr) + (int64_t)q * ldr) : (T)0;
      }
      __syncthreads();
      fold_panel(rows, p0);
    }
    cur = ls;
  }

  // Greedy column-pivoted QR of the b x b triangle (Definition 2.1 and the
  // remark after it): pivot = largest trailing column norm (recomputed each
  // step), ties to the lowest column; stop at |R_jj| <= eps |R_11|.
  for (int q = tid; q < b; q += NT) perm[q] = q;
  if (tid == 0) {
    s_k = b;
    s_r11 = (T)0;
  }
  __syncthreads();
  for (int j = 0; j < b; j++) {
    for (int cc = j + warp; cc < b; cc += nwarp) {
      const T *col = R + (int64_t)cc * ldr;
      T s = (T)0;
      for (int i = j + lane; i < b; i += 32) s += col[i] * col[i];
      s = warp_sum(s);
      if (lane == 0) nrm[cc] = s;
    }
    __syncthreads();
    if (warp == 0) {
      T best = (T)-1;
      int bi = b;
      for (int cc = j + lane; cc < b; cc += 32) {
        T v = nrm[cc];
        if (v > best) {
          best = v;
          bi = cc;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        T cn = sqrt(best);
        if (j == 0) s_r11 = cn;
        // no valid pivot (all norms NaN) also stops the factorization
        s_stop = (bi >= b || s_r11 == (T)0 || !(cn > (T)eps * s_r11)) ? 1 : 0;
        s_piv = bi;
        if (s_stop) s_k = j;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_piv;
    if (p != j) {
      for (int i = tid; i < b; i += NT) {
        T t0 = R[i + (int64_t)j * ldr];
        R[i + (int64_t)j * ldr] = R[i + (int64_t)p * ldr];
        R[i + (int64_t)p * ldr] = t0;
      }
      if (tid == 0) {
        int tp = perm[j];
        perm[j] = perm[p];
        perm[p] = tp;
      }
    }
    __syncthreads();
    {
      const T *cj = R + (int64_t)j * ldr;
      T s = (T)0;
      for (int i = j + 1 + lane; i < b; i += 32) s += cj[i] * cj[i];
      s = warp_sum(s);
      T x0 = cj[j];
      if (s > (T)0) {
        T nrm2 = sqrt(x0 * x0 + s);
        T beta = x0 >= (T)0 ? -nrm2 : nrm2;
        T tau = (beta - x0) / beta;
        T scl = (T)1 / (x0 - beta);
        for (int cc = j + 1 + warp; cc < b; cc += nwarp) {
          T *pc = R + (int64_t)cc * ldr;
          T d = (T)0;
          for (int i = j + 1 + lane; i < b; i += 32) d += cj[i] * pc[i];
          d = warp_sum(d);
          T wv = pc[j] + scl * d;
          T f = tau * wv;
          T fs = f * scl;
          for (int i = j + 1 + lane; i < b; i += 32) pc[i] -= fs * cj[i];
          __syncwarp();
          if (lane == 0) pc[j] -= f;
        }
      }
      __syncthreads();
      if (s > (T)0 && tid == 0) {
        T nrm2 = sqrt(x0 * x0 + s);
        R[j + (int64_t)j * ldr] = x0 >= (T)0 ? -nrm2 : nrm2;
      }
      __syncthreads();
    }
  }
  const int k = s_k;
  const int r = b - k;
  // T = R11^{-1} R12 by back substitution, one thread per column
  for (int cc = tid; cc < r; cc += NT) {
    T *tcol = fb.Tm + (int64_t)cc * k;
    for (int i = k - 1; i >= 0; i--) {
      T s = R[i + (int64_t)(k + cc) * ldr];
      for (int l = i + 1; l < k; l++) s -= R[i + (int64_t)l * ldr] * tcol[l];
      tcol[i] = s / R[i + (int64_t)i * ldr];
    }
  }
  for (int q = tid; q < b; q += NT) {
    fb.loc[q] = perm[q];
    fb.ids[q] = lv.cell_dofs[coff + perm[q]];
  }
  if (tid == 0) {
    fb.k = k;
    fb.r = r;
    fb.no = nO;
  }
}

constexpr unsigned FULL = 0xffffffffu;

// Rows of the ID matrix a thread keeps per panel column: 32 (FP32) / 16 (FP64).
template <typename T> struct IdwRows;
template <> struct IdwRows<float> { static constexpr int PR = 32; };
template <> struct IdwRows<double> { static constexpr int PR = 16; };

// ---------------------------------------------------------------------------
// Column-per-thread ID for boxes with b <= NC (64 or 128).  A "fold group" is
// NC threads; thread c owns column c of the group's b x b triangle R (shared
// memory, row-major) and holds column c of a PR-row panel of the ID matrix in
// registers.  One Householder reflector per column step: the owner of column
// j publishes it (and its squared norm) through a double buffer as soon as
// its update of step j-1 is done, the group synchronises on a named barrier,
// and every thread updates its own column.  G groups per box split the rows
// and their triangles are merged by a tree; group 0 then runs the greedy
// column-pivoted QR of the triangle, again one column per thread.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void group_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Vector loads and stores of a thread's panel rows (16-byte aligned
// addresses): float4 for FP32, double2 for FP64.
template <typename T, int N> __device__ __forceinline__ void store_vec(T *dst, const T (&v)[N]) {
  if constexpr (sizeof(T) == 4) {
    static_assert(N % 4 == 0, "FP32 rows in fours");
    float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int i = 0; i < N / 4; i++) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else {
    static_assert(N % 2 == 0, "FP64 rows in pairs");
    double2 *d2 = reinterpret_cast<double2 *>(dst);
#pragma unroll
    for (int i = 0; i < N / 2; i++) d2[i] = make_double2(v[2 * i], v[2 * i + 1]);
  }
}
template <typename T, int N> __device__ __forceinline__ void load_vec(T (&v)[N], const T *src) {
  if constexpr (sizeof(T) == 4) {
    static_assert(N % 4 == 0, "FP32 rows in fours");
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int i = 0; i < N / 4; i++) {
      const float4 t = s4[i];
      v[4 * i] = t.x;
      v[4 * i + 1] = t.y;
      v[4 * i + 2] = t.z;
      v[4 * i + 3] = t.w;
    }
  } else {
    static_assert(N % 2 == 0, "FP64 rows in pairs");
    const double2 *s2 = reinterpret_cast<const double2 *>(src);
#pragma unroll
    for (int i = 0; i < N / 2; i++) {
      const double2 t = s2[i];
      v[2 * i] = t.x;
      v[2 * i + 1] = t.y;
    }
  }
}

// Sums and updates over a thread's panel rows.  FP32 goes through the
// paired FMA (__ffma2_rn: two correctly rounded FMAs per instruction) with
// the same grouping of partial sums as the scalar form, so both give the
// same bits; FP64 stays scalar.
//   rows_dot8:   sum_i v_i p_i over eight interleaved partial sums
//   rows_dot2:   the same over two
//   rows_sumsq4: sum_i p_i^2 over four
//   rows_sumsq2: the same over two
//   rows_axpy:   p_i -= f v_i
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

template <typename T, int N> __device__ __forceinline__ T rows_dot8(const T (&v)[N], const T (&p)[N]) {
  if constexpr (sizeof(T) == 4 && N % 8 == 0) {
    float2 d[4];
#pragma unroll
    for (int u = 0; u < 4; u++) d[u] = f2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < N; i += 8)
#pragma unroll
      for (int u = 0; u < 4; u++)
        d[u] = __ffma2_rn(f2(v[i + 2 * u], v[i + 2 * u + 1]), f2(p[i + 2 * u], p[i + 2 * u + 1]), d[u]);
    return ((d[0].x + d[0].y) + (d[1].x + d[1].y)) + ((d[2].x + d[2].y) + (d[3].x + d[3].y));
  } else {
    T d[8];
#pragma unroll
    for (int u = 0; u < 8; u++) d[u] = (T)0;
#pragma unroll
    for (int i = 0; i < N; i += 8)
#pragma unroll
      for (int u = 0; u < 8 && i + u < N; u++) d[u] += v[i + u] * p[i + u];
    return ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7]));
  }
}
template <typename T, int N> __device__ __forceinline__ T rows_dot2(const T (&v)[N], const T (&p)[N]) {
  static_assert(N % 2 == 0, "rows in pairs");
  if constexpr (sizeof(T) == 4) {
    float2 d = f2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < N; i += 2) d = __ffma2_rn(f2(v[i], v[i + 1]), f2(p[i], p[i + 1]), d);
    return d.x + d.y;
  } else {
    T d0 = (T)0, d1 = (T)0;
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      d0 += v[i] * p[i];
      d1 += v[i + 1] * p[i + 1];
    }
    return d0 + d1;
  }
}
template <typename T, int N> __device__ __forceinline__ T rows_sumsq4(const T (&p)[N]) {
  static_assert(N % 4 == 0, "rows in fours");
  if constexpr (sizeof(T) == 4) {
    float2 s0 = f2(0.f, 0.f), s1 = f2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < N; i += 4) {
      s0 = __ffma2_rn(f2(p[i], p[i + 1]), f2(p[i], p[i + 1]), s0);
      s1 = __ffma2_rn(f2(p[i + 2], p[i + 3]), f2(p[i + 2], p[i + 3]), s1);
    }
    return (s0.x + s0.y) + (s1.x + s1.y);
  } else {
    T s0 = (T)0, s1 = (T)0, s2 = (T)0, s3 = (T)0;
#pragma unroll
    for (int i = 0; i < N; i += 4) {
      s0 += p[i] * p[i];
      s1 += p[i + 1] * p[i + 1];
      s2 += p[i + 2] * p[i + 2];
      s3 += p[i + 3] * p[i + 3];
    }
    return (s0 + s1) + (s2 + s3);
  }
}
template <typename T, int N> __device__ __forceinline__ T rows_sumsq2(const T (&p)[N]) {
  static_assert(N % 2 == 0, "rows in pairs");
  if constexpr (sizeof(T) == 4) {
    float2 s = f2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < N; i += 2) s = __ffma2_rn(f2(p[i], p[i + 1]), f2(p[i], p[i + 1]), s);
    return s.x + s.y;
  } else {
    T s0 = (T)0, s1 = (T)0;
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      s0 += p[i] * p[i];
      s1 += p[i + 1] * p[i + 1];
    }
    return s0 + s1;
  }
}
template <typename T, int N> __device__ __forceinline__ void rows_axpy(T (&p)[N], const T (&v)[N], T f) {
  if constexpr (sizeof(T) == 4 && N % 2 == 0) {
    const float2 nf = f2(-f, -f);
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const float2 r = __ffma2_rn(nf, f2(v[i], v[i + 1]), f2(p[i], p[i + 1]));
      p[i] = r.x;
      p[i + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) p[i] -= f * v[i];
  }
}

// The owner of column j publishes [v (PR entries) | tau | scl | beta | flag]
// for the reflector of step j, computed from its column, its squared norm
// and the current diagonal R[j][j]; flag = 0 means there is nothing to
// annihilate.  Entries are padded to a multiple of four for vector loads.
template <typename T, int PR>
__device__ __forceinline__ void publish_reflector(T *dst, const T (&pan)[PR], T x0) {
  const T s = rows_sumsq4<T, PR>(pan);
  store_vec<T, PR>(dst, pan);  // dst is 16-byte aligned: the buffers' stride is a multiple of 16 bytes
  if (s > (T)0) {
    const T nrm = sqrt(x0 * x0 + s);
    const T beta = x0 >= (T)0 ? -nrm : nrm;
    dst[PR] = (beta - x0) / beta;
    dst[PR + 1] = (T)1 / (x0 - beta);
    dst[PR + 2] = beta;
    dst[PR + 3] = (T)1;
  } else {
    dst[PR + 3] = (T)0;
  }
}

// Fold the PR rows in `pan` (this thread's column `col`) into R.  The
// reflector of step j is published by the owner of column j at the end of
// step j-1 (double buffer), so each step costs one barrier and, per thread,
// one vector load, a dot product and an update of its own column.
template <typename T, int PR>
__device__ __forceinline__ void fold_group(T (&pan)[PR], T *R, int ldr, int b, int col, T *vbuf, int bar_id,
                                           int nthr, int j0 = 0) {
  constexpr int VS = PR + 4;
  // j0 > 0: the panel is zero left of column j0 (rows j0.. of a triangle),
  // so the reflectors of the columns before it would change nothing
  if (col == j0 && j0 < b) publish_reflector<T, PR>(vbuf + (j0 & 1) * VS, pan, R[j0 * ldr + j0]);
  const int wlast = col | 31;  // the last column of this warp (columns of a warp are consecutive)
  T *Rj = R + (size_t)j0 * ldr;  // row j of the triangle
  for (int j = j0; j < b; j++, Rj += ldr) {
    group_bar(bar_id, nthr);
    if (j > wlast) continue;  // every column of this warp is done: only the barrier
    const T *vb = vbuf + (j & 1) * VS;
    if (vb[PR + 3] != (T)0) {  // the same for the whole group
      // every lane applies the reflector; columns at or left of j and
      // beyond b take f = 0, which leaves their rows as they are
      T v[PR];
      load_vec<T, PR>(v, vb);
      const T tau = vb[PR], scl = vb[PR + 1];
      const bool act = col > j && col < b;
      const T dd = rows_dot8<T, PR>(v, pan);
      const T rj = Rj[col];
      const T f = act ? tau * (rj + scl * dd) : (T)0;
      rows_axpy<T, PR>(pan, v, f * scl);
      if (act) Rj[col] = rj - f;
      else if (col == j) Rj[col] = vb[PR + 2];  // beta; nobody reads R[j][j] again in this fold
    }
    if (col == j + 1 && col < b) publish_reflector<T, PR>(vbuf + ((j + 1) & 1) * VS, pan, Rj[ldr + col]);
  }
  group_bar(bar_id, nthr);
}

template <int TPC> __device__ __forceinline__ unsigned col_mask() {
  return TPC == 1 ? 0xffffffffu : (((1u << TPC) - 1u) << ((threadIdx.x & 31) & ~(TPC - 1)));
}
template <typename T, int TPC> __device__ __forceinline__ T col_sum(T v) {
  const unsigned m = col_mask<TPC>();
#pragma unroll
  for (int o = 1; o < TPC; o <<= 1) v += __shfl_xor_sync(m, v, o);
  return v;
}

// Greedy column-pivoted QR of the box's b x b triangle R (row-major, ld
// LDR; GT = NC x TPC threads of the calling group, column `col` split over
// its TPC threads), T = R11^{-1} R12 and the box's ID outputs (Definition
// 2.1, with the pivot and truncation rule of the ID: largest trailing column
// norm, ties to the lowest column, k = #{j : |R_jj| > eps |R_11|}).
//   - Columns are not moved: each thread keeps the logical position of its
//     physical column, and the pivot's owner computes the reflector from its
//     own column, so a step costs two barriers (argmax, reflector).
//   - Trailing column norms are downdated (||x||^2 -= R_jc^2) and recomputed
//     from the column when they have lost half their digits (LAPACK's
//     safeguard); the pivot's own norm and the stopping test always use the
//     exact trailing norm.  In exact arithmetic the pivots are those of the
//     recomputed norms.
//   - T is formed in place (R12 := R11^{-1} R12) by back substitution, one
//     row of R11 per barrier with the updates spread over all threads, and
//     copied out coalesced.
template <typename T, int NC, int TPC> struct IdqShared {
  T red_v[16];
  int red_i[16], red_l[16];
  T hh[4];
  int lp[NC];  // physical column at each logical position
  int stop, k;
  T r11;
};

template <typename T, int NC, int TPC>
__device__ void idq_finish(T *R, int LDR, int b, double eps, int *perm, IdqShared<T, NC, TPC> &sh, FBox<T> &fb,
                           const LevelDev<T> &lv, int64_t coff, int nO) {
  constexpr int GT = NC * TPC;
  constexpr int NW = GT / 32;
  const int tid = threadIdx.x, lt = tid % GT, col = lt / TPC, part = lt % TPC;
  const int lane = tid & 31, wid = tid >> 5;
  // half the digits of T: recompute a norm once it has dropped below that
  const T tol = sizeof(T) == 4 ? (T)2.4e-4 : (T)1.5e-8;
  const bool own = col < b;
  int mylog = col;  // logical position of this thread's physical column
  // downdated and last exact trailing norms^2 of this thread's column
  T nrm = (T)0, nrm0 = (T)0;
  if (lt < b) perm[lt] = lt;
  if (own) {
    T a0 = (T)0;
    for (int i = part; i < b; i += TPC) a0 += R[i * LDR + col] * R[i * LDR + col];
    nrm = nrm0 = col_sum<T, TPC>(a0);
  }
  if (tid == 0) sh.k = b;
  // (largest norm, lowest logical position) over this warp's active columns
  auto warp_argmax = [&](int j) {
    T best = (T)-1;
    int bi = b, bl = b;
    if (own && part == 0 && mylog >= j) {
      best = nrm;
      bi = col;
      bl = mylog;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(FULL, best, o);
      const int oi = __shfl_xor_sync(FULL, bi, o), ol = __shfl_xor_sync(FULL, bl, o);
      if (ov > best || (ov == best && ol < bl)) {
        best = ov;
        bi = oi;
        bl = ol;
      }
    }
    if (lane == 0) {
      sh.red_v[wid] = best;
      sh.red_i[wid] = bi;
      sh.red_l[wid] = bl;
    }
  };
  group_bar(1, GT);
  warp_argmax(0);
  group_bar(1, GT);
  int j = 0;
  for (; j < b; j++) {
    // the pivot: every thread reduces the warps' candidates the same way
    T best = sh.red_v[0];
    int pc = sh.red_i[0], pl = sh.red_l[0];
    for (int u = 1; u < NW; u++)
      if (sh.red_v[u] > best || (sh.red_v[u] == best && sh.red_l[u] < pl)) {
        best = sh.red_v[u];
        pc = sh.red_i[u];
        pl = sh.red_l[u];
      }
    if (pc >= b) {  // no valid candidate (all norms NaN): stop
      if (tid == 0) sh.k = j;
      break;
    }
    if (col == pc) {
      // exact trailing norm of the pivot column, the stopping test and the
      // reflector (v = [1; R_(j+1..),pc scl], H = I - tau v v^T)
      T a0 = (T)0;
      for (int i = j + 1 + part; i < b; i += TPC) a0 += R[i * LDR + pc] * R[i * LDR + pc];
      const T sacc = col_sum<T, TPC>(a0);
      if (part == 0) {
        const T x0 = R[j * LDR + pc];
        const T cn = sqrt(x0 * x0 + sacc);
        if (j == 0) sh.r11 = cn;
        const T r11 = j == 0 ? cn : sh.r11;
        sh.stop = (r11 == (T)0 || !(cn > (T)eps * r11)) ? 1 : 0;
        if (sacc > (T)0) {
          const T beta = x0 >= (T)0 ? -cn : cn;
          sh.hh[1] = beta;
          sh.hh[2] = (beta - x0) / beta;
          sh.hh[3] = (T)1 / (x0 - beta);
        } else {
          sh.hh[2] = (T)0;  // tau = 0: nothing below the diagonal
        }
      }
    }
    // logical swap of positions j and pl (no data moves)
    if (mylog == j) mylog = pl;
    if (col == pc) mylog = j;
    if (tid == 0) {
      const int tp = perm[j];
      perm[j] = perm[pl];
      perm[pl] = tp;
    }
    group_bar(1, GT);
    if (sh.stop) {
      if (tid == 0) sh.k = j;
      break;
    }
    const T tau = sh.hh[2];
    if (own && mylog > j) {
      T rjc = R[j * LDR + col];
      if (tau != (T)0) {
        const T scl = sh.hh[3];
        T a0 = (T)0;
        for (int i = j + 1 + part; i < b; i += TPC) a0 += R[i * LDR + pc] * R[i * LDR + col];
        const T d = col_sum<T, TPC>(a0);
        const T f = tau * (rjc + scl * d);
        const T fs = f * scl;
        // eight rows at a time, loads before stores (the compiler cannot
        // tell that column col is not column pc)
        for (int i0 = j + 1 + part; i0 < b; i0 += 8 * TPC) {
          T xp[8], xc[8];
#pragma unroll
          for (int u = 0; u < 8; u++) {
            const int i = i0 + u * TPC;
            xp[u] = i < b ? R[i * LDR + pc] : (T)0;
            xc[u] = i < b ? R[i * LDR + col] : (T)0;
          }
#pragma unroll
          for (int u = 0; u < 8; u++) {
            const int i = i0 + u * TPC;
            if (i < b) R[i * LDR + col] = xc[u] - fs * xp[u];
          }
        }
        rjc -= f;
        if (part == 0) R[j * LDR + col] = rjc;
      }
      // row j leaves the trailing block of this column
      nrm -= rjc * rjc;
      if (!(nrm > tol * nrm0)) {
        T a0 = (T)0;
        for (int i = j + 1 + part; i < b; i += TPC) a0 += R[i * LDR + col] * R[i * LDR + col];
        nrm = nrm0 = col_sum<T, TPC>(a0);
      }
    }
    if (col == pc && part == 0 && tau != (T)0) R[j * LDR + pc] = sh.hh[1];
    warp_argmax(j + 1);
    group_bar(1, GT);
  }
  group_bar(1, GT);
  const int k = sh.k;
  const int r = b - k;
  if (own && part == 0) sh.lp[mylog] = col;
  group_bar(1, GT);
  // R12 := R11^{-1} R12 (columns of R12 are the logical positions k.. b-1)
  const FastDiv fr(max(r, 1)), fk(max(k, 1));
  for (int i = k - 1; i >= 0; i--) {
    const int pi = sh.lp[i];
    const T inv = (T)1 / R[i * LDR + pi];
    for (int c = lt; c < r; c += GT) R[i * LDR + sh.lp[k + c]] *= inv;
    group_bar(1, GT);
    for (int e = lt; e < i * r; e += GT) {
      int l, c;
      fr.divmod(e, l, c);
      const int pcol = sh.lp[k + c];
      R[l * LDR + pcol] -= R[l * LDR + pi] * R[i * LDR + pcol];
    }
    group_bar(1, GT);
  }
  // T (k x r, column-major, ld k)
  for (int e = lt; e < k * r; e += GT) {
    int i, c;
    fk.divmod(e, c, i);
    fb.Tm[e] = R[i * LDR + sh.lp[k + c]];
  }
  if (lt < b) {
    fb.loc[lt] = perm[lt];
    fb.ids[lt] = lv.cell_dofs[coff + perm[lt]];
  }
  if (tid == 0) {
    fb.k = k;
    fb.r = r;
    fb.no = nO;
  }
}

template <typename T, int NC, int RPT = IdwRows<T>::PR>
__global__ void __launch_bounds__(256) k_idc(LevelDev<T> lv, FBox<T> *boxes, const int *box_list, int nbox, int G,
                                             Points P, KernelParams K, ProxyParams px, const T *proxy_unit,
                                             double eps, int ring_max, int *err) {
  constexpr int PR = RPT;  // rows of a panel, all held by the column's thread
  constexpr int LDR = NC + 1;
  constexpr int VS = PR + 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ocode[125], s_obase[126], s_no;
  __shared__ IdqShared<T, NC, 1> s_sh;
  const int tid = threadIdx.x;
  const int grp = tid / NC, col = tid % NC;
  const int bar_id = 1 + grp;
  FBox<T> &fb = boxes[box_list[blockIdx.x]];
  const int c = fb.cell, b = fb.b, dim = lv.dim;
  T *Rg = reinterpret_cast<T *>(smem_raw) + (size_t)grp * NC * LDR;
  const size_t tri_bytes = (((size_t)G * NC * LDR * sizeof(T)) + 15) & ~(size_t)15;
  T *vbuf = reinterpret_cast<T *>(smem_raw + tri_bytes) + (size_t)grp * 2 * VS;
  int64_t *s_rowsrc = reinterpret_cast<int64_t *>(smem_raw + tri_bytes + (((size_t)G * 2 * VS * sizeof(T) + 15) & ~(size_t)15));
  int *perm = reinterpret_cast<int *>(s_rowsrc + ring_max);

  for (int e = col; e < NC * LDR; e += NC) Rg[e] = (T)0;
  if (tid < 32) {
    const int ncode = dim == 3 ? 125 : 25;
    int no = 0, acc = 0;
    for (int base = 0; base < ncode; base += 32) {
      int code = base + tid, cnt = 0;
      if (code < ncode) {
        int dx = code % 5 - 2, dy = (code / 5) % 5 - 2, dz = dim == 3 ? code / 25 - 2 : 0;
        const int dist = max(abs(dx), max(abs(dy), abs(dz)));
        if (dist == 2 || (lv.weak && dist == 1)) {  // ring O; weak steps: N too
          int nb = lv.cell_nbr[(int64_t)c * lv.NB + code];
          if (nb >= 0) cnt = lv.act_cnt[nb];
        }
      }
      unsigned mask = __ballot_sync(FULL, cnt > 0);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, incl, o);
        if (tid >= o) incl += t;
      }
      int pos = __popc(mask & ((1u << tid) - 1));
      if (cnt > 0) {
        s_ocode[no + pos] = code;
        s_obase[no + pos] = acc + incl - cnt;
      }
      no += __popc(mask);
      acc += __shfl_sync(FULL, incl, 31);
    }
    if (tid == 0) {
      s_obase[no] = acc;
      s_no = no;
    }
  }
  __syncthreads();
  const int no = s_no;
  const int nO = s_obase[no];
  if (nO > ring_max) {
    if (tid == 0) set_err(err, DERR_INTERNAL);
    return;  // uniform: every thread sees the same nO
  }
  for (int q = 0; q < no; q++) {
    const int code = s_ocode[q];
    const int nb = lv.cell_nbr[(int64_t)c * lv.NB + code];
    const int64_t abase = lv.cell_dof_off[nb];
    const int64_t pbase = lv.pair_off[(int64_t)c * lv.NB + code];
    for (int t = tid; t < s_obase[q + 1] - s_obase[q]; t += blockDim.x)
      s_rowsrc[s_obase[q] + t] = pbase + (int64_t)lv.act_idx[abase + t] * b;
  }
  __syncthreads();
  const int m = nO + px.np;
  const int64_t coff = lv.cell_dof_off[c];
  const double D = ldexp(1.0, -lv.t);
  const double rad = px.radius * D;
  // this column's point relative to the box centre, and the proxy radius, in
  // T: the proxy rows' distances take no FP64 arithmetic in the FP32 factor
  T xq[3];
  const T radT = (T)rad;
  {
    const int64_t g = col < b ? lv.cell_dofs[coff + col] : 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const double ctr = d < dim ? (lv.cell_coord[3 * c + d] + 0.5) * D : 0.0;
      xq[d] = (col < b && d < dim) ? (T)(P.x[g * dim + d] - ctr) : (T)0;
    }
  }
  const T w = (T)weight_of(P, K, lv.cell_dofs[lv.cell_dof_off[c]]);
  const int npan = (m + PR - 1) / PR;
  for (int pnl = grp; pnl < npan; pnl += G) {
    T pan[PR];
#pragma unroll
    for (int i = 0; i < PR; i++) {
      const int row = pnl * PR + i;
      T v = (T)0;
      if (col < b) {
        if (row < nO) {
          v = lv.pool[s_rowsrc[row] + col];
        } else if (row < m) {
          const int pm = row - nO;
          T r2 = (T)0;
#pragma unroll
          for (int d = 0; d < 3; d++) {
            const T dd = radT * proxy_unit[3 * pm + d] - xq[d];
            r2 += dd * dd;
          }
          v = w * kof(K.kind, r2);
        }
      }
      pan[i] = v;
    }
    fold_group<T, PR>(pan, Rg, LDR, b, col, vbuf, bar_id, NC);
  }
  // tree merge: in round `step`, group g (a multiple of 2*step) absorbs g + step
  for (int step = 1; step < G; step <<= 1) {
    __syncthreads();
    if (grp % (2 * step) == 0 && grp + step < G) {
      const T *Ro = Rg + (size_t)step * NC * LDR;
      for (int p0 = 0; p0 < b; p0 += PR) {
        T pan[PR];
#pragma unroll
        for (int i = 0; i < PR; i++) pan[i] = (p0 + i < b && col < b) ? Ro[(p0 + i) * LDR + col] : (T)0;
        fold_group<T, PR>(pan, Rg, LDR, b, col, vbuf, bar_id, NC, p0);
      }
    }
  }
  __syncthreads();
  if (grp != 0) return;
  idq_finish<T, NC, 1>(Rg, LDR, b, eps, perm, s_sh, fb, lv, coff, nO);
}

// ---------------------------------------------------------------------------
// The same column-per-thread ID with TPC threads per column and panels of
// PR = TPC x RPT rows: thread `part` of column c holds rows part*RPT .. +RPT
// of each panel, with the partial sums of a column combined by shuffles
// among its TPC lanes.  Each thread does the work per reflector step of
// k_idc, but a panel holds TPC times as many rows, so a box takes TPC times
// fewer sequential steps.  The reflectors, the triangle and the greedy
// pivoting are those of k_idc; only the order of partial sums differs.
// ---------------------------------------------------------------------------

// The TPC threads of the owner column publish [v (PR entries) | tau | scl |
// beta | flag] for the next reflector; see publish_reflector.
template <typename T, int PR, int TPC>
__device__ __forceinline__ void publish_part(T *dst, const T (&pan)[PR / TPC], T x0, int part) {
  constexpr int RPT = PR / TPC;
  const T s = col_sum<T, TPC>(rows_sumsq2<T, RPT>(pan));
  store_vec<T, RPT>(dst + part * RPT, pan);
  if (part == 0) {
    if (s > (T)0) {
      const T nrm = sqrt(x0 * x0 + s);
      const T beta = x0 >= (T)0 ? -nrm : nrm;
      dst[PR] = (beta - x0) / beta;
      dst[PR + 1] = (T)1 / (x0 - beta);
      dst[PR + 2] = beta;
      dst[PR + 3] = (T)1;
    } else {
      dst[PR + 3] = (T)0;
    }
  }
}

template <typename T, int PR, int TPC>
__device__ __forceinline__ void fold_group_q(T (&pan)[PR / TPC], T *R, int ldr, int b, int col, int part, T *vbuf,
                                             int bar_id, int nthr, int j0 = 0) {
  constexpr int VS = PR + 4, RPT = PR / TPC;
  // j0 > 0: the panel is zero left of column j0 (rows j0.. of a triangle)
  if (col == j0 && j0 < b) publish_part<T, PR, TPC>(vbuf + (j0 & 1) * VS, pan, R[j0 * ldr + j0], part);
  for (int j = j0; j < b; j++) {
    group_bar(bar_id, nthr);
    const T *vb = vbuf + (j & 1) * VS;
    T *vn = vbuf + ((j + 1) & 1) * VS;
    const T flag = vb[PR + 3];
    if (flag != (T)0) {
      if (col > j && col < b) {
        T v[RPT];
        load_vec<T, RPT>(v, vb + part * RPT);  // 16-byte aligned: VS and RPT are multiples of 4 (FP32) / 2 (FP64)
        const T tau = vb[PR], scl = vb[PR + 1];
        const T rj = R[j * ldr + col];
        const T dd = col_sum<T, TPC>(rows_dot2<T, RPT>(v, pan));  // also orders the read of rj before the write below
        const T f = tau * (rj + scl * dd);
        const T fs = f * scl;
        rows_axpy<T, RPT>(pan, v, fs);
        if (part == 0) R[j * ldr + col] = rj - f;
        if (col == j + 1) publish_part<T, PR, TPC>(vn, pan, R[col * ldr + col], part);
      } else if (col == j && part == 0) {
        R[j * ldr + j] = vb[PR + 2];
      }
    } else if (col == j + 1 && col < b) {
      publish_part<T, PR, TPC>(vn, pan, R[col * ldr + col], part);
    }
  }
  group_bar(bar_id, nthr);
}

template <typename T, int NC, int TPC>
__global__ void __launch_bounds__(512) k_idq(LevelDev<T> lv, FBox<T> *boxes, const int *box_list, int nbox, int G,
                                             Points P, KernelParams K, ProxyParams px, const T *proxy_unit,
                                             double eps, int ring_max, int *err) {
  constexpr int RPT = IdwRows<T>::PR;
  constexpr int PR = RPT * TPC;
  constexpr int VS = PR + 4;
  constexpr int GT = NC * TPC;  // threads per fold group
  static_assert(RPT % 2 == 0, "rows per thread");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ocode[125], s_obase[126], s_no;
  __shared__ IdqShared<T, NC, TPC> s_sh;
  const int tid = threadIdx.x;
  const int grp = tid / GT, lt = tid % GT;
  const int col = lt / TPC, part = lt % TPC;
  const int bar_id = 1 + grp;
  FBox<T> &fb = boxes[box_list[blockIdx.x]];
  const int c = fb.cell, b = fb.b, dim = lv.dim;
  // triangle rows x leading dimension: NC x (NC+1), or for the widest class
  // b x (b+1) (one group; shared memory sized by the level's widest box)
  const int TR = NC > 128 ? b : NC, LDR = TR + 1;
  T *Rg = reinterpret_cast<T *>(smem_raw) + (size_t)grp * TR * LDR;
  const size_t tri_bytes = (((size_t)G * TR * LDR * sizeof(T)) + 15) & ~(size_t)15;
  T *vbuf = reinterpret_cast<T *>(smem_raw + tri_bytes) + (size_t)grp * 2 * VS;
  int64_t *s_rowsrc =
      reinterpret_cast<int64_t *>(smem_raw + tri_bytes + (((size_t)G * 2 * VS * sizeof(T) + 15) & ~(size_t)15));
  int *perm = reinterpret_cast<int *>(s_rowsrc + ring_max);

  for (int e = lt; e < TR * LDR; e += GT) Rg[e] = (T)0;
  if (tid < 32) {
    const int ncode = dim == 3 ? 125 : 25;
    int no = 0, acc = 0;
    for (int base = 0; base < ncode; base += 32) {
      int code = base + tid, cnt = 0;
      if (code < ncode) {
        int dx = code % 5 - 2, dy = (code / 5) % 5 - 2, dz = dim == 3 ? code / 25 - 2 : 0;
        const int dist = max(abs(dx), max(abs(dy), abs(dz)));
        if (dist == 2 || (lv.weak && dist == 1)) {  // ring O; weak steps: N too
          int nb = lv.cell_nbr[(int64_t)c * lv.NB + code];
          if (nb >= 0) cnt = lv.act_cnt[nb];
        }
      }
      unsigned mask = __ballot_sync(FULL, cnt > 0);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, incl, o);
        if (tid >= o) incl += t;
      }
      int pos = __popc(mask & ((1u << tid) - 1));
      if (cnt > 0) {
        s_ocode[no + pos] = code;
        s_obase[no + pos] = acc + incl - cnt;
      }
      no += __popc(mask);
      acc += __shfl_sync(FULL, incl, 31);
    }
    if (tid == 0) {
      s_obase[no] = acc;
      s_no = no;
    }
  }
  __syncthreads();
  const int no = s_no;
  const int nO = s_obase[no];
  if (nO > ring_max) {
    if (tid == 0) set_err(err, DERR_INTERNAL);
    return;
  }
  for (int q = 0; q < no; q++) {
    const int code = s_ocode[q];
    const int nb = lv.cell_nbr[(int64_t)c * lv.NB + code];
    const int64_t abase = lv.cell_dof_off[nb];
    const int64_t pbase = lv.pair_off[(int64_t)c * lv.NB + code];
    for (int t = tid; t < s_obase[q + 1] - s_obase[q]; t += blockDim.x)
      s_rowsrc[s_obase[q] + t] = pbase + (int64_t)lv.act_idx[abase + t] * b;
  }
  __syncthreads();
  const int m = nO + px.np;
  const int64_t coff = lv.cell_dof_off[c];
  const double D = ldexp(1.0, -lv.t);
  const double rad = px.radius * D;
  // this column's point relative to the box centre, and the proxy radius, in
  // T: the proxy rows' distances take no FP64 arithmetic in the FP32 factor
  T xq[3];
  const T radT = (T)rad;
  {
    const int64_t g = col < b ? lv.cell_dofs[coff + col] : 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const double ctr = d < dim ? (lv.cell_coord[3 * c + d] + 0.5) * D : 0.0;
      xq[d] = (col < b && d < dim) ? (T)(P.x[g * dim + d] - ctr) : (T)0;
    }
  }
  const T w = (T)weight_of(P, K, lv.cell_dofs[lv.cell_dof_off[c]]);
  const int npan = (m + PR - 1) / PR;
  for (int pnl = grp; pnl < npan; pnl += G) {
    T pan[RPT];
#pragma unroll
    for (int i = 0; i < RPT; i++) {
      const int row = pnl * PR + part * RPT + i;
      T v = (T)0;
      if (col < b) {
        if (row < nO) {
          v = lv.pool[s_rowsrc[row] + col];
        } else if (row < m) {
          const int pm = row - nO;
          T r2 = (T)0;
#pragma unroll
          for (int d = 0; d < 3; d++) {
            const T dd = radT * proxy_unit[3 * pm + d] - xq[d];
            r2 += dd * dd;
          }
          v = w * kof(K.kind, r2);
        }
      }
      pan[i] = v;
    }
    fold_group_q<T, PR, TPC>(pan, Rg, LDR, b, col, part, vbuf, bar_id, GT);
  }
  for (int step = 1; step < G; step <<= 1) {
    __syncthreads();
    if (grp % (2 * step) == 0 && grp + step < G) {
      const T *Ro = Rg + (size_t)step * TR * LDR;
      for (int p0 = 0; p0 < b; p0 += PR) {
        T pan[RPT];
#pragma unroll
        for (int i = 0; i < RPT; i++) {
          const int row = p0 + part * RPT + i;
          pan[i] = (row < b && col < b) ? Ro[row * LDR + col] : (T)0;
        }
        fold_group_q<T, PR, TPC>(pan, Rg, LDR, b, col, part, vbuf, bar_id, GT, p0);
      }
    }
  }
  __syncthreads();
  if (grp != 0) return;
  idq_finish<T, NC, TPC>(Rg, LDR, b, eps, perm, s_sh, fb, lv, coff, nO);
}

// ---------------------------------------------------------------------------
// One box's ID over C CTAs (for colour phases with few boxes): CTA `chunk`
// folds panels chunk, chunk + C, ... of the box's ID matrix into its own
// triangle (as k_idq with one group), writes it to its slot of `tri`, and
// the slots are merged pairwise up a binary tree.  At each tree node a
// counter tells the second CTA of the pair to arrive that it merges: it
// holds (or loads) the left triangle and folds the right one's rows into it,
// so the result does not depend on arrival order; the first to arrive exits.
// The CTA that completes the root runs the pivoted QR and writes the ID.
// No CTA waits for another.
// ---------------------------------------------------------------------------
template <typename T, int NC, int TPC, bool GLOB>
__global__ void __launch_bounds__(512) k_idm(LevelDev<T> lv, FBox<T> *boxes, const int *box_list, int C, Points P,
                                             KernelParams K, ProxyParams px, const T *proxy_unit, double eps,
                                             int ring_max, T *tri, int64_t tstride, int *cnt, int *err) {
  constexpr int RPT = IdwRows<T>::PR;
  constexpr int PR = RPT * TPC;
  constexpr int VS = PR + 4;
  constexpr int GT = NC * TPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ocode[125], s_obase[126], s_no, s_second;
  __shared__ int64_t s_pbase[125], s_abase[125];  // GLOB: each ring cell's pair block and active list
  __shared__ IdqShared<T, NC, TPC> s_sh;
  const int tid = threadIdx.x, lt = tid;
  const int col = lt / TPC, part = lt % TPC;
  const int bq = blockIdx.x / C, chunk = blockIdx.x % C;
  FBox<T> &fb = boxes[box_list[bq]];
  const int c = fb.cell, b = fb.b, dim = lv.dim;
  const int TR = NC > 128 ? b : NC, LDR = TR + 1;
  // the triangle in shared memory, or (GLOB: boxes too wide for it) in this
  // CTA's slot of `tri`, where it stays L2-resident: the fold touches one row
  // of it per reflector step
  T *slots = tri + (int64_t)bq * C * tstride;
  T *R = GLOB ? slots + (int64_t)chunk * tstride : reinterpret_cast<T *>(smem_raw);
  const size_t tri_bytes = GLOB ? 0 : (((size_t)TR * LDR * sizeof(T)) + 15) & ~(size_t)15;
  T *vbuf = reinterpret_cast<T *>(smem_raw + tri_bytes);
  int64_t *s_rowsrc = reinterpret_cast<int64_t *>(smem_raw + tri_bytes + (((size_t)2 * VS * sizeof(T) + 15) & ~(size_t)15));
  int *perm = reinterpret_cast<int *>(s_rowsrc + (GLOB ? 0 : ring_max));

  for (int e = lt; e < TR * LDR; e += GT) R[e] = (T)0;
  if (tid < 32) {
    const int ncode = dim == 3 ? 125 : 25;
    int no = 0, acc = 0;
    for (int base = 0; base < ncode; base += 32) {
      int code = base + tid, cnt_ = 0;
      if (code < ncode) {
        int dx = code % 5 - 2, dy = (code / 5) % 5 - 2, dz = dim == 3 ? code / 25 - 2 : 0;
        const int dist = max(abs(dx), max(abs(dy), abs(dz)));
        if (dist == 2 || (lv.weak && dist == 1)) {  // ring O; weak steps: N too
          int nb = lv.cell_nbr[(int64_t)c * lv.NB + code];
          if (nb >= 0) cnt_ = lv.act_cnt[nb];
        }
      }
      unsigned mask = __ballot_sync(FULL, cnt_ > 0);
      int incl = cnt_;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, incl, o);
        if (tid >= o) incl += t;
      }
      int pos = __popc(mask & ((1u << tid) - 1));
      if (cnt_ > 0) {
        s_ocode[no + pos] = code;
        s_obase[no + pos] = acc + incl - cnt_;
      }
      no += __popc(mask);
      acc += __shfl_sync(FULL, incl, 31);
    }
    if (tid == 0) {
      s_obase[no] = acc;
      s_no = no;
    }
  }
  __syncthreads();
  const int no = s_no;
  const int nO = s_obase[no];
  if (nO > ring_max) {
    if (tid == 0) set_err(err, DERR_INTERNAL);
    return;  // every CTA of the box sees the same nO: the box's tree is abandoned whole
  }
  if (GLOB) {
    for (int q = tid; q < no; q += blockDim.x) {
      const int code = s_ocode[q];
      s_abase[q] = lv.cell_dof_off[lv.cell_nbr[(int64_t)c * lv.NB + code]];
      s_pbase[q] = lv.pair_off[(int64_t)c * lv.NB + code];
    }
  } else {
    for (int q = 0; q < no; q++) {
      const int code = s_ocode[q];
      const int nb = lv.cell_nbr[(int64_t)c * lv.NB + code];
      const int64_t abase = lv.cell_dof_off[nb];
      const int64_t pbase = lv.pair_off[(int64_t)c * lv.NB + code];
      for (int t = tid; t < s_obase[q + 1] - s_obase[q]; t += blockDim.x)
        s_rowsrc[s_obase[q] + t] = pbase + (int64_t)lv.act_idx[abase + t] * b;
    }
  }
  __syncthreads();
  // pool offset of ring row `row` (< nO): the table, or (GLOB) its ring cell
  // by binary search over the cells' first rows
  auto rowsrc = [&](int row) -> int64_t {
    if (!GLOB) return s_rowsrc[row];
    int lo = 0, hi = no - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_obase[mid] <= row) lo = mid;
      else hi = mid - 1;
    }
    return s_pbase[lo] + (int64_t)lv.act_idx[s_abase[lo] + (row - s_obase[lo])] * b;
  };
  const int m = nO + px.np;
  const int64_t coff = lv.cell_dof_off[c];
  const double D = ldexp(1.0, -lv.t);
  const double rad = px.radius * D;
  // this column's point relative to the box centre, and the proxy radius, in
  // T: the proxy rows' distances take no FP64 arithmetic in the FP32 factor
  T xq[3];
  const T radT = (T)rad;
  {
    const int64_t g = col < b ? lv.cell_dofs[coff + col] : 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const double ctr = d < dim ? (lv.cell_coord[3 * c + d] + 0.5) * D : 0.0;
      xq[d] = (col < b && d < dim) ? (T)(P.x[g * dim + d] - ctr) : (T)0;
    }
  }
  const T w = (T)weight_of(P, K, lv.cell_dofs[lv.cell_dof_off[c]]);
  const int npan = (m + PR - 1) / PR;
  for (int pnl = chunk; pnl < npan; pnl += C) {
    T pan[RPT];
#pragma unroll
    for (int i = 0; i < RPT; i++) {
      const int row = pnl * PR + part * RPT + i;
      T v = (T)0;
      if (col < b) {
        if (row < nO) {
          v = lv.pool[rowsrc(row) + col];
        } else if (row < m) {
          const int pm = row - nO;
          T r2 = (T)0;
#pragma unroll
          for (int d = 0; d < 3; d++) {
            const T dd = radT * proxy_unit[3 * pm + d] - xq[d];
            r2 += dd * dd;
          }
          v = w * kof(K.kind, r2);
        }
      }
      pan[i] = v;
    }
    fold_group_q<T, PR, TPC>(pan, R, LDR, b, col, part, vbuf, 1, GT);
  }
  int cur = chunk;  // first slot of the subtree this CTA carries
  for (int L = 1; L < C; L <<= 1) {
    const int ls = cur & ~(2 * L - 1), rs = ls + L;
    if (rs >= C) continue;  // no right partner at this level: carry the subtree up
    // publish this subtree's triangle, then count arrivals at the node
    if (!GLOB) {
      T *mine = slots + (int64_t)cur * tstride;
      for (int e = lt; e < TR * LDR; e += GT) mine[e] = R[e];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      int *node = cnt + ((int64_t)bq * 8 + (31 - __clz(L))) * C + ls;
      const int seen = atomicAdd(node, 1);
      s_second = seen == 1;
      if (seen == 1) *node = 0;  // reset for the next launch
    }
    __syncthreads();
    if (!s_second) return;
    __threadfence();
    if (cur != ls) {  // came from the right: continue on the left triangle
      T *left = slots + (int64_t)ls * tstride;
      if (GLOB) {
        R = left;
      } else {
        for (int e = lt; e < TR * LDR; e += GT) R[e] = __ldcg(left + e);
      }
      __syncthreads();
    }
    const T *right = slots + (int64_t)rs * tstride;
    for (int p0 = 0; p0 < b; p0 += PR) {
      T pan[RPT];
#pragma unroll
      for (int i = 0; i < RPT; i++) {
        const int row = p0 + part * RPT + i;
        pan[i] = (row < b && col < b) ? __ldcg(right + row * LDR + col) : (T)0;
      }
      fold_group_q<T, PR, TPC>(pan, R, LDR, b, col, part, vbuf, 1, GT, p0);
    }
    cur = ls;
  }
  __syncthreads();
  idq_finish<T, NC, TPC>(R, LDR, b, eps, perm, s_sh, fb, lv, coff, nO);
}

template <typename T, int NC, int TPC, bool GLOB = false>
static size_t idm_smem(int bmax, int ring_max) {
  constexpr int PR = IdwRows<T>::PR * TPC;
  const int TR = NC > 128 ? bmax : NC;
  return (GLOB ? 0 : ((((size_t)TR * (TR + 1) * sizeof(T)) + 15) & ~(size_t)15)) +
         ((((size_t)2 * (PR + 4) * sizeof(T)) + 15) & ~(size_t)15) + (GLOB ? 0 : (size_t)ring_max * sizeof(int64_t)) +
         (size_t)NC * sizeof(int) + 16;
}

template <typename T, int NC, int TPC, bool GLOB = false>
static void launch_idm(const LevelDev<T> &lv, FBox<T> *boxes, const int *box_list, int nbox, int C, int bmax,
                       const Points &P, const KernelParams &K, const ProxyParams &px, const T *proxy_unit,
                       double eps, int ring_max, T *tri, int64_t tstride, int *cnt, cudaStream_t st, int *err) {
  const size_t smem = idm_smem<T, NC, TPC, GLOB>(bmax, ring_max);
  cudaFuncSetAttribute(k_idm<T, NC, TPC, GLOB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_idm<T, NC, TPC, GLOB><<<nbox * C, NC * TPC, smem, st>>>(lv, boxes, box_list, C, P, K, px, proxy_unit, eps,
                                                            ring_max, tri, tstride, cnt, err);
  count_launch();
}

// Shared memory of a k_idq launch (see the kernel's layout).
template <typename T, int NC, int TPC> static size_t idq_smem(int bmax, int G, int ring_max) {
  constexpr int PR = IdwRows<T>::PR * TPC;
  const int TR = NC > 128 ? bmax : NC;
  const size_t tri = (size_t)TR * (TR + 1) * sizeof(T);
  return (((size_t)G * tri + 15) & ~(size_t)15) + (((size_t)G * 2 * (PR + 4) * sizeof(T) + 15) & ~(size_t)15) +
         (size_t)ring_max * sizeof(int64_t) + (size_t)NC * sizeof(int) + 16;
}

template <typename T, int NC, int TPC>
static void launch_idq(const LevelDev<T> &lv, FBox<T> *boxes, const int *box_list, int nbox, int G, int bmax,
                       const Points &P, const KernelParams &K, const ProxyParams &px, const T *proxy_unit,
                       double eps, int ring_max, cudaStream_t st, int *err) {
  constexpr int PR = IdwRows<T>::PR * TPC;
  const int TR = NC > 128 ? bmax : NC;
  const size_t tri = (size_t)TR * (TR + 1) * sizeof(T);
  int gmax = (int)((190u << 10) / tri);
  if (gmax < 1) gmax = 1;
  if (G > gmax) G = gmax;
  if (G * NC * TPC > 512) G = 512 / (NC * TPC);
  if (G < 1) G = 1;
  (void)PR;
  const size_t smem = idq_smem<T, NC, TPC>(bmax, G, ring_max);
  cudaFuncSetAttribute(k_idq<T, NC, TPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_idq<T, NC, TPC><<<nbox, G * NC * TPC, smem, st>>>(lv, boxes, box_list, nbox, G, P, K, px, proxy_unit, eps,
                                                      ring_max, err);
  count_launch();
}

template <typename T, int NC, int RPT = IdwRows<T>::PR>
static void launch_idc(const LevelDev<T> &lv, FBox<T> *boxes, const int *box_list, int nbox, int G,
                       const Points &P, const KernelParams &K, const ProxyParams &px, const T *proxy_unit,
                       double eps, int ring_max, cudaStream_t st, int *err) {
  constexpr int PR = RPT;
  const size_t tri = (size_t)NC * (NC + 1) * sizeof(T);
  int gmax = (int)((190u << 10) / tri);
  if (gmax < 1) gmax = 1;
  if (G > gmax) G = gmax;
  if (G * NC > 256) G = 256 / NC;
  size_t smem = (((size_t)G * tri + 15) & ~(size_t)15) + (((size_t)G * 2 * (PR + 4) * sizeof(T) + 15) & ~(size_t)15) +
                (size_t)ring_max * sizeof(int64_t) + (size_t)NC * sizeof(int) + 16;
  cudaFuncSetAttribute(k_idc<T, NC, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_idc<T, NC, RPT><<<nbox, G * NC, smem, st>>>(lv, boxes, box_list, nbox, G, P, K, px, proxy_unit, eps, ring_max,
                                                err);
  count_launch();
}


// ---------------------------------------------------------------------------
// Warp-per-panel ID for boxes with b <= 64 (k_idw), the panels pipelined
// into one triangle.  One CTA of W warps per box; warp w folds row panels
// w, w + W, ... of the ID matrix.  Lane l keeps columns l and l + 32 of a
// PR-row panel in registers and the reflector of each step goes through the
// warp's own buffer in shared memory (a __syncwarp, not a barrier across
// warps, orders it).  All warps fold into the same b x b triangle: panel p
// takes step j one iteration after panel p - 1 took it, since step j reads
// and writes only row j of the triangle, which panel p - 1 finished at its
// own step j.  In one iteration the warps work on different rows, a barrier
// over the CTA separates iterations, and warp w runs W iterations behind
// nobody: panel w starts at iteration w, panel w + W one round (max(b, W)
// iterations) later.  No triangle per warp and no merge: ceil(panels / W)
// rounds of b steps, then all W warps run the column-pivoted QR of the
// triangle (idq_finish, W / 2 threads per column).  Reflectors, triangle
// and pivoting are those of k_idc; only the order in which rows are folded
// and partial sums are added differs.
// ---------------------------------------------------------------------------

// Apply the reflector (v, tau, scl) of the current step to one column: its
// PR panel rows `p` and its entry of the triangle's current row, *rjc.
template <typename T, int PR>
__device__ __forceinline__ void warp_col_update(T (&p)[PR], const T (&v)[PR], T tau, T scl, T *rjc) {
  const T dd = rows_dot8<T, PR>(v, p);
  const T rj = *rjc;
  const T f = tau * (rj + scl * dd);
  const T fs = f * scl;
  rows_axpy<T, PR>(p, v, fs);
  *rjc = rj - f;
}

// Step j of a warp's panel (column lane + 32 s in slot s of p): the owner
// of column j publishes the reflector from its column and R[j][j], then
// every lane applies it to its columns right of j and row j of R.
template <typename T, int PR, int NS>
__device__ __forceinline__ void warp_step(T (&p)[NS][PR], T *R, int ldr, int b, int lane, T *vb, int j) {
  if constexpr (NS == 2) {  // the slot is uniform over the warp: no selects
    if (j < 32) {
      if (lane == j) publish_reflector<T, PR>(vb, p[0], R[j * ldr + j]);
    } else if (lane == j - 32) {
      publish_reflector<T, PR>(vb, p[1], R[j * ldr + j]);
    }
  } else if (lane == (j & 31)) {
    // the owner's column j, picked from its slots with static indices (so
    // that the panel stays in registers)
    const int js = j >> 5;
    T src[PR];
#pragma unroll
    for (int i = 0; i < PR; i++) {
      src[i] = p[0][i];
#pragma unroll
      for (int sl = 1; sl < NS; sl++)
        if (js == sl) src[i] = p[sl][i];
    }
    publish_reflector<T, PR>(vb, src, R[j * ldr + j]);
  }
  __syncwarp();
  if (vb[PR + 3] != (T)0) {
    T v[PR];
    load_vec<T, PR>(v, vb);
    const T tau = vb[PR], scl = vb[PR + 1];
#pragma unroll
    for (int sl = 0; sl < NS; sl++) {
      const int c = lane + 32 * sl;
      if (j < 32 * sl + 31 && c > j && c < b) warp_col_update<T, PR>(p[sl], v, tau, scl, R + j * ldr + c);
    }
    if (lane == (j & 31)) R[j * ldr + j] = vb[PR + 2];  // later panels read the new R[j][j]
  }
  __syncwarp();  // the buffer is written again at the next step
}

// Rows per panel of the warp-per-panel ID: 32 (FP32) / 16 (FP64) for 64
// columns (two per lane), half that for 128 (four per lane).
template <typename T, int NC> struct IdpRows {
  static constexpr int PR = NC == 64 ? IdwRows<T>::PR : IdwRows<T>::PR / 2;
};

template <typename T, int W, int NC>
__global__ void __launch_bounds__(W * 32) k_idw(LevelDev<T> lv, FBox<T> *boxes, const int *box_list, Points P,
                                                KernelParams K, ProxyParams px, const T *proxy_unit, double eps,
                                                int ring_max, int *err) {
  constexpr int PR = IdpRows<T, NC>::PR;
  constexpr int NS = NC / 32;  // columns per lane
  constexpr int LDR = NC + 1;
  constexpr int VS = PR + 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ocode[125], s_obase[126], s_no;
  __shared__ IdqShared<T, NC, W * 32 / NC> s_sh;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  FBox<T> &fb = boxes[box_list[blockIdx.x]];
  const int c = fb.cell, b = fb.b, dim = lv.dim;
  T *R = reinterpret_cast<T *>(smem_raw);
  const size_t tri_bytes = (((size_t)NC * LDR * sizeof(T)) + 15) & ~(size_t)15;
  T *vb = reinterpret_cast<T *>(smem_raw + tri_bytes) + (size_t)wid * VS;
  int64_t *s_rowsrc =
      reinterpret_cast<int64_t *>(smem_raw + tri_bytes + (((size_t)W * VS * sizeof(T) + 15) & ~(size_t)15));
  int *perm = reinterpret_cast<int *>(s_rowsrc + ring_max);

  for (int e = tid; e < NC * LDR; e += W * 32) R[e] = (T)0;
  if (tid < 32) {
    const int ncode = dim == 3 ? 125 : 25;
    int no = 0, acc = 0;
    for (int base = 0; base < ncode; base += 32) {
      int code = base + tid, cnt = 0;
      if (code < ncode) {
        int dx = code % 5 - 2, dy = (code / 5) % 5 - 2, dz = dim == 3 ? code / 25 - 2 : 0;
        const int dist = max(abs(dx), max(abs(dy), abs(dz)));
        if (dist == 2 || (lv.weak && dist == 1)) {  // ring O; weak steps: N too
          int nb = lv.cell_nbr[(int64_t)c * lv.NB + code];
          if (nb >= 0) cnt = lv.act_cnt[nb];
        }
      }
      unsigned mask = __ballot_sync(FULL, cnt > 0);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, incl, o);
        if (tid >= o) incl += t;
      }
      int pos = __popc(mask & ((1u << tid) - 1));
      if (cnt > 0) {
        s_ocode[no + pos] = code;
        s_obase[no + pos] = acc + incl - cnt;
      }
      no += __popc(mask);
      acc += __shfl_sync(FULL, incl, 31);
    }
    if (tid == 0) {
      s_obase[no] = acc;
      s_no = no;
    }
  }
  __syncthreads();
  const int no = s_no;
  const int nO = s_obase[no];
  if (nO > ring_max) {
    if (tid == 0) set_err(err, DERR_INTERNAL);
    return;  // uniform: every thread sees the same nO
  }
  for (int q = 0; q < no; q++) {
    const int code = s_ocode[q];
    const int nb = lv.cell_nbr[(int64_t)c * lv.NB + code];
    const int64_t abase = lv.cell_dof_off[nb];
    const int64_t pbase = lv.pair_off[(int64_t)c * lv.NB + code];
    for (int t = tid; t < s_obase[q + 1] - s_obase[q]; t += blockDim.x)
      s_rowsrc[s_obase[q] + t] = pbase + (int64_t)lv.act_idx[abase + t] * b;
  }
  __syncthreads();
  const int m = nO + px.np;
  const int64_t coff = lv.cell_dof_off[c];
  const double D = ldexp(1.0, -lv.t);
  const double rad = px.radius * D;
  // the lane's points relative to the box centre, and the proxy radius, in
  // T: the proxy rows' distances take no FP64 arithmetic in the FP32 factor
  T xq[NS][3];
  const T radT = (T)rad;
#pragma unroll
  for (int sl = 0; sl < NS; sl++) {
    const int col = lane + 32 * sl;
    const int64_t g = col < b ? lv.cell_dofs[coff + col] : 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const double ctr = d < dim ? (lv.cell_coord[3 * c + d] + 0.5) * D : 0.0;
      xq[sl][d] = (col < b && d < dim) ? (T)(P.x[g * dim + d] - ctr) : (T)0;
    }
  }
  const T w = (T)weight_of(P, K, lv.cell_dofs[lv.cell_dof_off[c]]);
  const int npan = (m + PR - 1) / PR;
  const int L = max(b, W);  // iterations per round of W panels
  const int iters = ((npan + W - 1) / W) * L + W - 1;
  T p[NS][PR];
  for (int it = 0; it < iters; it++) {
    group_bar(1, W * 32);
    const int local = it - wid;
    if (local < 0) continue;
    const int j = local % L, pnl = wid + (local / L) * W;
    if (pnl >= npan || j >= b) continue;
    if (j == 0) {  // this warp's next panel
#pragma unroll
      for (int i = 0; i < PR; i++) {
        const int row = pnl * PR + i;
        if (row < nO) {
          const int64_t src = s_rowsrc[row];
#pragma unroll
          for (int sl = 0; sl < NS; sl++) {
            const int col = lane + 32 * sl;
            p[sl][i] = col < b ? lv.pool[src + col] : (T)0;
          }
        } else if (row < m) {
          const int pm = row - nO;
          T u[3];
#pragma unroll
          for (int d = 0; d < 3; d++) u[d] = radT * proxy_unit[3 * pm + d];
#pragma unroll
          for (int sl = 0; sl < NS; sl++) {
            T r2 = (T)0;
#pragma unroll
            for (int d = 0; d < 3; d++) r2 += (u[d] - xq[sl][d]) * (u[d] - xq[sl][d]);
            p[sl][i] = lane + 32 * sl < b ? w * kof(K.kind, r2) : (T)0;
          }
        } else {
#pragma unroll
          for (int sl = 0; sl < NS; sl++) p[sl][i] = (T)0;
        }
      }
    }
    warp_step<T, PR, NS>(p, R, LDR, b, lane, vb, j);
  }
  __syncthreads();
  idq_finish<T, NC, W * 32 / NC>(R, LDR, b, eps, perm, s_sh, fb, lv, coff, nO);
}

template <typename T, int W, int NC> static size_t idw_smem(int ring_max) {
  constexpr int PR = IdpRows<T, NC>::PR;
  return ((((size_t)NC * (NC + 1) * sizeof(T)) + 15) & ~(size_t)15) +
         ((((size_t)W * (PR + 4) * sizeof(T)) + 15) & ~(size_t)15) + (size_t)ring_max * sizeof(int64_t) +
         NC * sizeof(int) + 16;
}

template <typename T, int W, int NC>
static bool launch_idw(const LevelDev<T> &lv, FBox<T> *boxes, const int *box_list, int nbox, const Points &P,
                       const KernelParams &K, const ProxyParams &px, const T *proxy_unit, double eps,
                       int ring_max, cudaStream_t st, int *err) {
  const size_t smem = idw_smem<T, W, NC>(ring_max);
  if (smem > (size_t)(220u << 10)) return false;  // a ring too long for the row table
  cudaFuncSetAttribute(k_idw<T, W, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_idw<T, W, NC><<<nbox, W * 32, smem, st>>>(lv, boxes, box_list, P, K, px, proxy_unit, eps, ring_max, err);
  count_launch();
  return true;
}

// Launch shape of the next ID launch on this thread: fold groups per box
// (hint & 15), threads per column ((hint >> 4) & 15; 0 or 1: k_idc), CTAs
// per box ((hint >> 8) & 15; more than 1: k_idm), with bit 12 set the
// warp-per-panel kernel k_idw with 2^(hint & 15) warps, with bit 13 set
// (k_idc) twice the panel rows per thread; 0: default.  Set by the host's
// autotuner around a launch_id call, with the multi-CTA scratch.
static thread_local int id_groups_hint = 0;
static thread_local IdMultiScratch id_multi{};
void set_id_groups(int G) { id_groups_hint = G; }
void set_id_multi(const IdMultiScratch &m) { id_multi = m; }

template <typename T>
void launch_id(const LevelDev<T> &lv, FBox<T> *boxes, const int *box_list, int nbox, int bmax, int mmax,
               const Points &P, const KernelParams &K, const ProxyParams &px, const T *proxy_unit, double eps,
               T *gscratch, int64_t gscratch_stride, bool use_smem, cudaStream_t st, int *err) {
  (void)mmax;
  if (nbox == 0) return;
  const bool force_general = bmax < 0;  // large-box path requested
  if (force_general) bmax = -bmax;
  if (bmax <= 128 && !force_general) {
    const int ring_max = mmax;
    // fold groups per box: the autotuner's choice for this (precision, box
    // width, phase size), else the default (enough boxes resident at once to
    // finish a large phase in one wave, more groups per box when small)
    const int NCw = bmax <= 64 ? 64 : 128;
    if (((id_groups_hint >> 12) & 1) && NCw == 64) {  // warp per panel: 2^(hint & 15) warps
      const int W = 1 << (id_groups_hint & 15);
      bool done = false;
      if (W == 2) done = launch_idw<T, 2, 64>(lv, boxes, box_list, nbox, P, K, px, proxy_unit, eps, ring_max, st, err);
      else if (W == 4) done = launch_idw<T, 4, 64>(lv, boxes, box_list, nbox, P, K, px, proxy_unit, eps, ring_max, st, err);
      else if (W == 8) done = launch_idw<T, 8, 64>(lv, boxes, box_list, nbox, P, K, px, proxy_unit, eps, ring_max, st, err);
      if (done) return;
    }
    int G = id_groups_hint & 15, TPC = (id_groups_hint >> 4) & 15, C = (id_groups_hint >> 8) & 15;
    const int64_t ts = (int64_t)NCw * (NCw + 1);
    if (C > 1 && TPC >= 2 && id_multi.tri && (int64_t)nbox * C <= id_multi.max_slots && ts <= id_multi.slot_elems &&
        NCw * TPC <= 512) {
      if (NCw == 64) {
        if (TPC == 4) launch_idm<T, 64, 4>(lv, boxes, box_list, nbox, C, bmax, P, K, px, proxy_unit, eps, ring_max, (T *)id_multi.tri, ts, id_multi.cnt, st, err);
        else launch_idm<T, 64, 2>(lv, boxes, box_list, nbox, C, bmax, P, K, px, proxy_unit, eps, ring_max, (T *)id_multi.tri, ts, id_multi.cnt, st, err);
      } else {
        if (TPC == 4) launch_idm<T, 128, 4>(lv, boxes, box_list, nbox, C, bmax, P, K, px, proxy_unit, eps, ring_max, (T *)id_multi.tri, ts, id_multi.cnt, st, err);
        else launch_idm<T, 128, 2>(lv, boxes, box_list, nbox, C, bmax, P, K, px, proxy_unit, eps, ring_max, (T *)id_multi.tri, ts, id_multi.cnt, st, err);
      }
      return;
    }
    if (G <= 0) G = NCw == 64 ? (nbox >= 300 ? 2 : 4) : (nbox >= 300 ? 1 : 2);
    if (TPC <= 0) TPC = 1;
    // bit 13: one thread per column holding twice the rows of a panel
    constexpr int R2 = 2 * IdwRows<T>::PR;
    const bool rows2 = TPC == 1 && ((id_groups_hint >> 13) & 1);
    if (NCw == 64) {
      if (TPC == 4) launch_idq<T, 64, 4>(lv, boxes, box_list, nbox, G, bmax, P, K, px, proxy_unit, eps, ring_max, st, err);
      else if (TPC == 2) launch_idq<T, 64, 2>(lv, boxes, box_list, nbox, G, bmax, P, K, px, proxy_unit, eps, ring_max, st, err);
      else if (rows2) launch_idc<T, 64, R2>(lv, boxes, box_list, nbox, G, P, K, px, proxy_unit, eps, ring_max, st, err);
      else launch_idc<T, 64>(lv, boxes, box_list, nbox, G, P, K, px, proxy_unit, eps, ring_max, st, err);
    } else {
      if (TPC == 4) launch_idq<T, 128, 4>(lv, boxes, box_list, nbox, G, bmax, P, K, px, proxy_unit, eps, ring_max, st, err);
      else if (TPC == 2) launch_idq<T, 128, 2>(lv, boxes, box_list, nbox, G, bmax, P, K, px, proxy_unit, eps, ring_max, st, err);
      else if (rows2) launch_idc<T, 128, R2>(lv, boxes, box_list, nbox, G, P, K, px, proxy_unit, eps, ring_max, st, err);
      else launch_idc<T, 128>(lv, boxes, box_list, nbox, G, P, K, px, proxy_unit, eps, ring_max, st, err);
    }
    return;
  }
  if (bmax <= 256 && !force_general) {
    // one group per box, the triangle sized by the level's widest box
    const int TPC = ((id_groups_hint >> 4) & 15) == 1 ? 1 : 2, C = (id_groups_hint >> 8) & 15;
    if (C > 1 && TPC == 2 && id_multi.tri && (int64_t)nbox * C <= id_multi.max_slots &&
        (int64_t)bmax * (bmax + 1) <= id_multi.slot_elems) {
      const size_t smw = (((size_t)bmax * (bmax + 1) * sizeof(T) + 15) & ~(size_t)15) + 2 * (64 + 4) * sizeof(T) + 16 +
                         (size_t)mmax * sizeof(int64_t) + 256 * sizeof(int) + 16;
      if (smw <= (size_t)(220 << 10)) {
        launch_idm<T, 256, 2>(lv, boxes, box_list, nbox, C, bmax, P, K, px, proxy_unit, eps, mmax, (T *)id_multi.tri,
                              (int64_t)bmax * (bmax + 1), id_multi.cnt, st, err);
        return;
      }
    }
    const size_t sm = TPC == 1 ? idq_smem<T, 256, 1>(bmax, 1, mmax) : idq_smem<T, 256, 2>(bmax, 1, mmax);
    if (sm <= (size_t)(220 << 10)) {
      if (TPC == 1) launch_idq<T, 256, 1>(lv, boxes, box_list, nbox, 1, bmax, P, K, px, proxy_unit, eps, mmax, st, err);
      else launch_idq<T, 256, 2>(lv, boxes, box_list, nbox, 1, bmax, P, K, px, proxy_unit, eps, mmax, st, err);
      return;
    }
  }
  if (bmax <= 512 && !force_general) {
    // boxes too wide for a shared-memory triangle: several CTAs per box
    // with their triangles in global (L2-resident) slots
    const int C = ((id_groups_hint >> 8) & 15) > 1 ? ((id_groups_hint >> 8) & 15) : 16;  // 8: 904 ms, 16: 827 ms (3D 32^3, 1e-6)
    if (id_multi.tri && (int64_t)nbox * C <= id_multi.max_slots &&
        (int64_t)bmax * (bmax + 1) <= id_multi.slot_elems &&
        idm_smem<T, 512, 1, true>(bmax, mmax) <= (size_t)(220 << 10)) {
      launch_idm<T, 512, 1, true>(lv, boxes, box_list, nbox, C, bmax, P, K, px, proxy_unit, eps, mmax,
                                  (T *)id_multi.tri, (int64_t)bmax * (bmax + 1), id_multi.cnt, st, err);
      return;
    }
  }
  int PR = bmax <= 80 ? 128 : 64;
  IdLayout<T> lay(bmax, PR);
  size_t smem = use_smem ? (size_t)lay.bytes : 0;
  if (use_smem)
    cudaFuncSetAttribute(k_id<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // several CTAs per box (workspaces in global memory, the level's
  // scratch holding C of them per box), one for the forced large-box path
  int C = 1;
  if (!use_smem && !force_general && id_multi.kid_ctas > 1 && id_multi.cnt &&
      (int64_t)nbox * id_multi.kid_ctas <= id_multi.max_slots)
    C = id_multi.kid_ctas;
  if (C > 1) {  // the panel in shared memory: PR rows (ld PR + 1) x bmax columns
    PR = sizeof(T) == 4 ? 32 : 16;
    while (PR > 8 && (size_t)(PR + 1) * bmax * sizeof(T) > (size_t)(200 << 10)) PR /= 2;
    smem = (size_t)(PR + 1) * bmax * sizeof(T) + 16;
    if (smem > (size_t)(220 << 10)) {  // too wide even for 8-row panels: one CTA per box
      C = 1;
      PR = bmax <= 80 ? 128 : 64;
      smem = 0;
    } else {
      cudaFuncSetAttribute(k_id<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
  }
  k_id<T><<<nbox * C, NT, smem, st>>>(lv, boxes, box_list, P, K, px, eps, PR, gscratch, gscratch_stride,
                                      use_smem ? 1 : 0, C, id_multi.cnt, err); count_launch();
}

template <typename T> int64_t id_region_bytes(int b, int PR) { return IdLayout<T>(b, PR).bytes; }
template int64_t id_region_bytes<float>(int, int);
template int64_t id_region_bytes<double>(int, int);

// ---------------------------------------------------------------------------
// Elimination of the redundant DOFs (Sec. 3.1, Eq. 3.4)
// ---------------------------------------------------------------------------

// Storage for the box's LU, X_RR^{-1} (r x r each), E and G (nj x r each)
// (run by one thread, before any of them is written): the host's reservation
// when the rank the ID found and the box's |J| fit it, else a slice of the
// level's overflow space.  When neither has room the box records
// DERR_CAPACITY, eliminates nothing (r = 0, so the Schur launch skips it) and
// the host redoes the factorization with full-size reservations.
template <typename T>
__device__ bool claim_storage(FBox<T> &fb, int nj, const Overflow<T> &ov, int *err) {
  const int r = fb.r;
  if (r <= fb.rres && (int64_t)nj * r <= (int64_t)fb.njres * fb.rres) return true;
  const bool symm = fb.G == nullptr;  // symmetric storage: no G
  const int64_t need = (2 * (int64_t)r * r + (symm ? 1 : 2) * (int64_t)nj * r + 3) & ~int64_t(3);
  if (ov.cap > 0) {
    const unsigned long long o = atomicAdd(ov.used, (unsigned long long)need);
    if ((int64_t)o + need <= ov.cap) {
      T *p = ov.base + o;
      fb.LU = p;
      p += (int64_t)r * r;
      fb.Xi = p;
      p += (int64_t)r * r;
      fb.E = p;
      p += (int64_t)nj * r;
      fb.G = symm ? nullptr : p;
      return true;
    }
  }
  set_err(err, DERR_CAPACITY);
  fb.k = fb.b;
  fb.r = 0;
  return false;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_elim(LevelDev<T> lv, FBox<T> *boxes, const int *box_list, T *scratch,
                                             int64_t sstride, int64_t ws_off, Overflow<T> ovf, int *err, int C,
                                             int form_only) {
  __shared__ int s_ncode[27], s_ncell[27], s_nstart[28], s_nn;
  __shared__ int64_t s_off_in[27], s_off_out[27];
  __shared__ int s_ld_in[27];
  __shared__ int s_pivrow, s_ok;

  // C CTAs per box: every CTA forms its share of the rows of X_JR and columns
  // of X_RJ; CTA 0 also forms the S columns of X_RJ (the X_RS its LU needs)
  // and, unless form_only (X_RR, its LU and inverse then follow in
  // k_elim_xrr and k_elim_lu), the LU, X_RR^{-1} and the box's records
  const int q = blockIdx.x / C, cta = blockIdx.x % C;
  FBox<T> &fb = boxes[box_list[q]];
  const int c = fb.cell, b = fb.b, k = fb.k, r = fb.r, dim = lv.dim;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = NT / 32;
  const int ncode3 = dim == 3 ? 27 : 9;
  const int center = code3(0, 0, 0, dim);

  // T (k x r, ld k) and loc (b ints) read from the box's records in place
  // (every CTA of the box reads them); the LU (r x r, ld r+1) and the pivots
  // (r ints) in this box's global workspace, written by CTA 0 only
  T *LU = scratch + (int64_t)q * sstride + ws_off;
  const int ldl = r + 1;
  const T *Ts = fb.Tm;
  const int *sloc = fb.loc;
  int *spiv = reinterpret_cast<int *>(LU + (int64_t)r * ldl);

  if (tid == 0) {
    int nn = 0, acc = k;
    for (int code = 0; code < ncode3; code++) {
      int dx, dy, dz;
      decode3(code, dim, dx, dy, dz);
      int nb = lv.cell_nbr[(int64_t)c * lv.NB + code5(dx, dy, dz, dim)];
      s_ncell[code] = nb;
      if (nb >= 0) {
        s_off_in[code] = lv.pair_off[(int64_t)nb * lv.NB + code5(-dx, -dy, -dz, dim)];
        s_off_out[code] = lv.pair_off[(int64_t)c * lv.NB + code5(dx, dy, dz, dim)];
        s_ld_in[code] = lv.cell_b[nb];
      }
      if (code == center || nb < 0 || lv.weak) continue;  // weak steps: J = S
      int cnt = lv.act_cnt[nb];
      if (cnt <= 0) continue;
      s_ncode[nn] = code;
      s_nstart[nn] = acc;
      acc += cnt;
      nn++;
    }
    s_nstart[nn] = acc;
    s_nn = nn;
    s_ok = (acc <= fb.njmax && cta == 0) ? claim_storage(fb, acc, ovf, err) : 1;  // acc > njmax: reported below
  }
  __syncthreads();
  if (!s_ok) return;
  const int nn = s_nn;
  const int nj = s_nstart[nn];
  if (nj > fb.njmax) {
    if (tid == 0) set_err(err, DERR_INTERNAL);
    return;
  }
  // J = [S (pivot order); N (near cells in code order, active ascending)]
  for (int a = tid; a < nj; a += NT) {
    int code, loc;
    int64_t g;
    if (a < k) {
      code = center;
      loc = sloc[a];
      g = fb.ids[a];
    } else {
      int q = 0;
      while (s_nstart[q + 1] <= a) q++;
      code = s_ncode[q];
      int nb = s_ncell[code];
      loc = lv.act_idx[lv.cell_dof_off[nb] + (a - s_nstart[q])];
      g = lv.cell_dofs[lv.cell_dof_off[nb] + loc];
    }
    if (cta == 0) {
      fb.J[a] = g;
      fb.Jnb[a] = code;
      fb.Jloc[a] = loc;
    }
  }
  if (tid == 0 && cta == 0) fb.nj = nj;
  __syncthreads();
  // (3^d code, local index) of J entry a, as in the J lists above
  auto jinfo = [&](int a, int &code, int &la) {
    if (a < k) {
      code = center;
      la = sloc[a];
    } else {
      int q2 = 0;
      while (s_nstart[q2 + 1] <= a) q2++;
      code = s_ncode[q2];
      la = lv.act_idx[lv.cell_dof_off[s_ncell[code]] + (a - s_nstart[q2])];
    }
  };

  T *Ep = scratch + (int64_t)q * sstride;  // X_JR, nj x r col-major (ld nj)
  T *Gp = Ep + (int64_t)nj * r;                      // X_RJ, r x nj col-major (ld r)
  const T *pool = lv.pool;
  const T *Aii = pool + s_off_in[center];            // block (c, c), ld b

  // X_JR = A_JR - A_JS T   (L_T applied from the right)
  for (int a = cta * NT + tid; a < nj; a += C * NT) {
    int code, la;
    jinfo(a, code, la);
    const T *Ab = pool + s_off_in[code];
    int64_t ld = s_ld_in[code];
    const T *row = Ab + la;
    for (int r0 = 0; r0 < r; r0 += 8) {
      T acc[8];
#pragma unroll
      for (int u = 0; u < 8; u++) acc[u] = (r0 + u < r) ? row[(int64_t)sloc[k + r0 + u] * ld] : (T)0;
      for (int s = 0; s < k; s++) {
        T as = row[(int64_t)sloc[s] * ld];
#pragma unroll
        for (int u = 0; u < 8; u++)
          if (r0 + u < r) acc[u] -= as * Ts[s + (int64_t)(r0 + u) * k];
      }
#pragma unroll
      for (int u = 0; u < 8; u++)
        if (r0 + u < r) Ep[a + (int64_t)(r0 + u) * nj] = acc[u];
    }
  }
  // X_RJ = A_RJ - T^T A_SJ  (U_T applied from the left); one warp per column:
  // the S columns by CTA 0, the others shared by all CTAs
  auto xrj_col = [&](int a) {
    int code, la;
    jinfo(a, code, la);
    const T *col = pool + s_off_out[code] + (int64_t)la * b;  // column la of block (c, nb)
    for (int ri = lane; ri < r; ri += 32) {
      T acc = col[sloc[k + ri]];
      for (int s = 0; s < k; s++) acc -= Ts[s + (int64_t)ri * k] * col[sloc[s]];
      Gp[ri + (int64_t)a * r] = acc;
    }
  };
  if (cta == 0)
    for (int a = warp; a < k; a += nwarp) xrj_col(a);
  for (int a = k + cta * nwarp + warp; a < nj; a += C * nwarp) xrj_col(a);
  __syncthreads();
  if (cta != 0 || form_only) return;
  // X_RR = A_RR - T^T A_SR - X_RS T   (X_RS = first k columns of X_RJ)
  for (int e = tid; e < r * r; e += NT) {
    int ri = e / r, rj = e % r;
    int64_t qc = (int64_t)sloc[k + rj] * b;
    T acc = Aii[sloc[k + ri] + qc];
    for (int s = 0; s < k; s++) {
      acc -= Ts[s + (int64_t)ri * k] * Aii[sloc[s] + qc];
      acc -= Gp[ri + (int64_t)s * r] * Ts[s + (int64_t)rj * k];
    }
    LU[ri * ldl + rj] = acc;
  }
  for (int i = tid; i < r; i += NT) spiv[i] = i;
  __syncthreads();
  // LU with partial pivoting (largest |entry|, ties to the lowest row)
  for (int j = 0; j < r; j++) {
    if (warp == 0) {
      T best = (T)-1;
      int bi = r;
      for (int i = j + lane; i < r; i += 32) {
        T v = fabs(LU[i * ldl + j]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        if (bi >= r) {  // NaN column: keep the diagonal, report
          bi = j;
          set_err(err, DERR_NUMERIC);
        }
        s_pivrow = bi;
        if (best == (T)0) set_err(err, DERR_NUMERIC);
      }
    }
    __syncthreads();
    const int p = s_pivrow;
    if (p != j) {
      for (int cc = tid; cc < r; cc += NT) {
        T t0 = LU[j * ldl + cc];
        LU[j * ldl + cc] = LU[p * ldl + cc];
        LU[p * ldl + cc] = t0;
      }
      if (tid == 0) {
        int tp = spiv[j];
        spiv[j] = spiv[p];
        spiv[p] = tp;
      }
    }
    __syncthreads();
    const T d = LU[j * ldl + j];
    for (int i = j + 1 + tid; i < r; i += NT) LU[i * ldl + j] /= d;
    __syncthreads();
    const int rem = r - j - 1;
    for (int e = tid; e < rem * rem; e += NT) {
      int i = j + 1 + e / rem, cc = j + 1 + e % rem;
      LU[i * ldl + cc] -= LU[i * ldl + j] * LU[j * ldl + cc];
    }
    __syncthreads();
  }
  // E = X_JR X_RR^{-1} and G = X_RR^{-1} X_RJ follow in k_elim_gemm, over
  // every box of the phase at once, from X_JR, X_RJ (scratch) and X_RR^{-1}
  for (int e = tid; e < r * r; e += NT) fb.LU[e] = LU[(e / r) * ldl + (e % r)];
  for (int i = tid; i < r; i += NT) fb.piv[i] = spiv[i];
  // X_RR^{-1} = U^{-1} L^{-1} P, one column per thread (column piv[i] is
  // U^{-1} L^{-1} e_i), kept for the solve sweeps
  for (int i0 = tid; i0 < r; i0 += NT) {
    T *x = fb.Xi + (int64_t)spiv[i0] * r;
    for (int i = 0; i < r; i++) {
      T sacc = i == i0 ? (T)1 : (T)0;
      for (int l = 0; l < i; l++) sacc -= LU[i * ldl + l] * x[l];
      x[i] = sacc;
    }
    for (int i = r - 1; i >= 0; i--) {
      T sacc = x[i];
      for (int l = i + 1; l < r; l++) sacc -= LU[i * ldl + l] * x[l];
      x[i] = sacc / LU[i * ldl + i];
    }
  }
  // the box's active DOFs are now its skeleton, kept in ascending order
  const int64_t coff = lv.cell_dof_off[c];
  for (int s = tid; s < k; s += NT) {
    int v = sloc[s], rank = 0;
    for (int s2 = 0; s2 < k; s2++) rank += sloc[s2] < v;
    lv.act_idx[coff + rank] = v;
  }
  if (tid == 0) lv.act_cnt[c] = k;
}

// ---------------------------------------------------------------------------
// Elimination, shared-memory form for b small enough: the LU of X_RR is
// formed by the whole CTA, one rank-1 update per column (warp 0 picks each
// pivot), X_RR^{-1} = U^{-1} L^{-1} P column by column from the LU factors
// (a thread per column), and E = X_JR X_RR^{-1},
// G = X_RR^{-1} X_RJ are produced in chunks of CH rows / columns of J as
// shared-memory products, written coalesced.  X_RJ is kept in the scratch
// for the Schur update.
// ---------------------------------------------------------------------------

// C (m x n) = A (m x K) B (K x n) from shared memory, 256 threads as 16 x 16
// with an MX x NY register tile each (a 16 MX x 16 NY block per pass);
// A(i,l) = A[i*sai + l*sal], B(l,j) = B[l + j*sbj] (B is contiguous along
// l); each result goes to out(i, j, value).  A's unit stride (AU = 1: sai
// is 1, AU = 2: sal is 1) is a template argument so that the loads of a
// thread address one register plus constant offsets.  In single precision
// pairs of columns share one paired FMA (two correctly rounded FMAs, so the
// sums are those of the scalar form: l ascending, one fused multiply-add
// per term).
template <typename T, int MX, int NY, int AU, typename Out>
__device__ __forceinline__ void smem_gemm_blk(int m, int n, int K, const T *A, int sai_, int sal_, const T *B,
                                              int sbj, Out out) {
  static_assert(AU == 1 || AU == 2, "A must be unit-stride along i or l");
  const int sai = AU == 1 ? 1 : sai_, sal = AU == 2 ? 1 : sal_, sbl = 1;
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
  for (int i0 = 0; i0 < m; i0 += 16 * MX)
    for (int j0 = 0; j0 < n; j0 += 16 * NY) {
      bool rv[MX], cv[NY];
#pragma unroll
      for (int x = 0; x < MX; x++) rv[x] = i0 + ti + 16 * x < m;
#pragma unroll
      for (int y = 0; y < NY; y++) cv[y] = j0 + tj + 16 * y < n;
      // rows and columns past the matrix read row / column 0 (their
      // products are never stored), so the loads need no predicate
      const T *ap[MX], *bp[NY];
#pragma unroll
      for (int x = 0; x < MX; x++) ap[x] = A + (rv[x] ? (i0 + ti + 16 * x) * sai : 0);
#pragma unroll
      for (int y = 0; y < NY; y++) bp[y] = B + (cv[y] ? (j0 + tj + 16 * y) * sbj : 0);
      T acc[MX][NY];
      if constexpr (std::is_same<T, float>::value && NY % 2 == 0) {
        float2 a2[MX][NY / 2];
#pragma unroll
        for (int x = 0; x < MX; x++)
#pragma unroll
          for (int y = 0; y < NY / 2; y++) a2[x][y] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int l = 0; l < K; l++) {
          float a[MX], bb[NY];
#pragma unroll
          for (int x = 0; x < MX; x++) a[x] = ap[x][l * sal];
#pragma unroll
          for (int y = 0; y < NY; y++) bb[y] = bp[y][l * sbl];
#pragma unroll
          for (int x = 0; x < MX; x++)
#pragma unroll
            for (int y = 0; y < NY / 2; y++)
              a2[x][y] = __ffma2_rn(make_float2(a[x], a[x]), make_float2(bb[2 * y], bb[2 * y + 1]), a2[x][y]);
        }
#pragma unroll
        for (int x = 0; x < MX; x++)
#pragma unroll
          for (int y = 0; y < NY / 2; y++) {
            acc[x][2 * y] = a2[x][y].x;
            acc[x][2 * y + 1] = a2[x][y].y;
          }
      } else {
#pragma unroll
        for (int x = 0; x < MX; x++)
#pragma unroll
          for (int y = 0; y < NY; y++) acc[x][y] = (T)0;
#pragma unroll 4
        for (int l = 0; l < K; l++) {
          T a[MX], bb[NY];
#pragma unroll
          for (int x = 0; x < MX; x++) a[x] = ap[x][l * sal];
#pragma unroll
          for (int y = 0; y < NY; y++) bb[y] = bp[y][l * sbl];
#pragma unroll
          for (int x = 0; x < MX; x++)
#pragma unroll
            for (int y = 0; y < NY; y++) acc[x][y] += a[x] * bb[y];
        }
      }
#pragma unroll
      for (int x = 0; x < MX; x++)
#pragma unroll
        for (int y = 0; y < NY; y++)
          if (rv[x] && cv[y]) out(i0 + ti + 16 * x, j0 + tj + 16 * y, acc[x][y]);
    }
}

// The block shape (32 x 64 or 64 x 32) that covers m x n in fewer passes;
// every call of a CTA takes the same branch (m, n are uniform).
template <typename T, int AU, typename Out>
__device__ __forceinline__ void smem_gemm(int m, int n, int K, const T *A, int sai, int sal, const T *B, int sbj,
                                          Out out) {
  const int p24 = ((m + 31) >> 5) * ((n + 63) >> 6), p42 = ((m + 63) >> 6) * ((n + 31) >> 5);
  if (p42 < p24)
    smem_gemm_blk<T, 4, 2, AU>(m, n, K, A, sai, sal, B, sbj, out);
  else
    smem_gemm_blk<T, 2, 4, AU>(m, n, K, A, sai, sal, B, sbj, out);
}

template <typename T> struct ElimChunk;
template <> struct ElimChunk<float> { static constexpr int CH = 32; };
template <> struct ElimChunk<double> { static constexpr int CH = 32; };

template <typename T>
__host__ __device__ inline size_t elim2_smem(int b, int k, int r) {
  constexpr int CH = ElimChunk<T>::CH;
  const int ldx = r | 1;
  size_t pers = (size_t)k * r * 3 + (size_t)r * (r + 1);
  size_t u1 = (size_t)b * (b + 1);
  size_t u2 = (size_t)ldx * r + (size_t)(CH + 1) * b + (size_t)(b + 1) * CH;
  size_t nT = pers + (u1 > u2 ? u1 : u2);
  return nT * sizeof(T) + (size_t)(b + 2 * r + 8) * sizeof(int) + 64;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_elim2(LevelDev<T> lv, FBox<T> *boxes, const int *box_list, T *scratch,
                                              int64_t sstride, Overflow<T> ovf, int *err, int split, int C) {
  constexpr int CH = ElimChunk<T>::CH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ncode[27], s_ncell[27], s_nstart[28], s_nact[27], s_nn, s_ok;
  __shared__ int64_t s_off_in[27], s_off_out[27];
  __shared__ int s_ld_in[27];
  __shared__ int64_t s_rb[ElimChunk<T>::CH], s_cb[ElimChunk<T>::CH];
  __shared__ int s_rl[ElimChunk<T>::CH];
  // C CTAs per box (split mode only): CTA 0 also does the LU, X_RR^{-1} and
  // the box's records; every CTA forms its share of the chunks of J
  const int q = blockIdx.x / C, cta = blockIdx.x % C;
  FBox<T> &fb = boxes[box_list[q]];
  const int c = fb.cell, b = fb.b, k = fb.k, r = fb.r, dim = lv.dim;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ncode3 = dim == 3 ? 27 : 9;
  const int center = code3(0, 0, 0, dim);
  const int ldx = r | 1, ldl = r + 1, ldb = b + 1;
  T *Ts = reinterpret_cast<T *>(smem_raw);          // k x r  (s + ri*k)
  T *XRS = Ts + (size_t)k * r;                      // r x k  (ri + s*r)
  T *XSR = XRS + (size_t)k * r;                     // k x r  (s + ri*k)
  T *LU = XSR + (size_t)k * r;                      // r x r row-major, ld r+1
  T *U0 = LU + (size_t)r * ldl;                     // union region
  T *Ab = U0;                                       // A_BB in (S|R) order, column-major, ld b+1
  T *Xi = U0;                                       // X_RR^{-1}, column-major, ld ldx (after the LU)
  T *rawJ = Xi + (size_t)ldx * r;                   // CH rows of J x b  (al + p*(CH+1)) -> X_JR in place
  T *rawC = rawJ + (size_t)(CH + 1) * b;            // b x CH columns of J (p + al*(b+1)) -> X_RJ in place
  const size_t u1 = (size_t)b * ldb, u2 = (size_t)ldx * r + (size_t)(CH + 1) * b + (size_t)ldb * CH;
  int *sloc = reinterpret_cast<int *>(U0 + (u1 > u2 ? u1 : u2));
  int *spiv = sloc + b;
  int *spinv = spiv + r;

  if (tid == 0) {
    int nn = 0, acc = k;
    for (int code = 0; code < ncode3; code++) {
      int dx, dy, dz;
      decode3(code, dim, dx, dy, dz);
      int nb = lv.cell_nbr[(int64_t)c * lv.NB + code5(dx, dy, dz, dim)];
      s_ncell[code] = nb;
      if (nb >= 0) {
        s_off_in[code] = lv.pair_off[(int64_t)nb * lv.NB + code5(-dx, -dy, -dz, dim)];
        s_off_out[code] = lv.pair_off[(int64_t)c * lv.NB + code5(dx, dy, dz, dim)];
        s_ld_in[code] = lv.cell_b[nb];
      }
      if (code == center || nb < 0 || lv.weak) continue;  // weak steps: J = S
      int cnt = lv.act_cnt[nb];
      if (cnt <= 0) continue;
      s_ncode[nn] = code;
      s_nstart[nn] = acc;
      s_nact[nn] = (int)lv.cell_dof_off[nb];
      acc += cnt;
      nn++;
    }
    s_nstart[nn] = acc;
    s_nn = nn;
    s_ok = (acc <= fb.njmax && cta == 0) ? claim_storage(fb, acc, ovf, err) : 1;  // acc > njmax: reported below
  }
  for (int q = tid; q < b; q += NT) sloc[q] = fb.loc[q];
  for (int e = tid; e < k * r; e += NT) Ts[e] = fb.Tm[e];
  __syncthreads();
  if (!s_ok) return;
  const int nn = s_nn;
  const int nj = s_nstart[nn];
  if (nj > fb.njmax) {
    if (tid == 0) set_err(err, DERR_INTERNAL);
    return;
  }
  // J = [S (pivot order); N (near cells in code order, active ascending)]
  for (int a = tid; a < nj; a += NT) {
    int code, loc;
    int64_t g;
    if (a < k) {
      code = center;
      loc = sloc[a];
      g = fb.ids[a];
    } else {
      int q = 0;
      while (s_nstart[q + 1] <= a) q++;
      code = s_ncode[q];
      loc = lv.act_idx[s_nact[q] + (a - s_nstart[q])];
      g = lv.cell_dofs[s_nact[q] + loc];
    }
    if (cta == 0) {
      fb.J[a] = g;
      fb.Jnb[a] = code;
      fb.Jloc[a] = loc;
    }
  }
  if (tid == 0 && cta == 0) fb.nj = nj;
  // stage A_BB in (S|R) order
  const FastDiv fdb(max(b, 1)), fdr(max(r, 1)), fdk(max(k, 1));
  const T *Aii = lv.pool + s_off_in[center];
  for (int e = tid; e < b * b; e += NT) {
    int pp, qq;
    fdb.divmod(e, qq, pp);
    Ab[pp + qq * ldb] = Aii[sloc[pp] + (int64_t)sloc[qq] * b];
  }
  __syncthreads();
  // X_RS = A_RS - T^T A_SS,  X_SR = A_SR - A_SS T,  then
  // X_RR = A_RR - T^T A_SR - X_RS T (all as tiled shared-memory products)
  for (int e = tid; e < r * k; e += NT) {
    int ri, s2;
    fdr.divmod(e, s2, ri);
    XRS[ri + s2 * r] = Ab[(k + ri) + s2 * ldb];
  }
  for (int e = tid; e < r * k; e += NT) {
    int s2, ri;
    fdk.divmod(e, ri, s2);
    XSR[s2 + ri * k] = Ab[s2 + (k + ri) * ldb];
  }
  for (int e = tid; e < r * r; e += NT) {
    int ri, rj;
    fdr.divmod(e, rj, ri);
    LU[ri * ldl + rj] = Ab[(k + ri) + (k + rj) * ldb];
  }
  __syncthreads();
  {
    T *xrs = XRS, *xsr = XSR, *lu = LU;
    const int rr = r, kk = k, ll = ldl;
    smem_gemm<T, 2>(r, k, k, Ts, k, 1, Ab, ldb, [&](int ri, int s2, T v) { xrs[ri + s2 * rr] -= v; });
    smem_gemm<T, 1>(k, r, k, Ab, 1, ldb, Ts, k, [&](int s2, int ri, T v) { xsr[s2 + ri * kk] -= v; });
    smem_gemm<T, 2>(r, r, k, Ts, k, 1, Ab + (size_t)k * ldb, ldb, [&](int ri, int rj, T v) { lu[ri * ll + rj] -= v; });
  }
  __syncthreads();
  {
    T *lu = LU;
    const int ll = ldl;
    smem_gemm<T, 1>(r, r, k, XRS, 1, r, Ts, k, [&](int ri, int rj, T v) { lu[ri * ll + rj] -= v; });
  }
  __syncthreads();
  if (cta == 0) {
  // LU with partial pivoting (largest |entry|, ties to the lowest row): per
  // column, warp 0 picks the pivot, swaps the rows and scales the column;
  // then every warp takes rows of the rank-1 update, its lanes 32
  // consecutive columns
  for (int i = tid; i < r; i += NT) spiv[i] = i;
  __syncthreads();
  for (int j = 0; j < r; j++) {
    if (warp == 0) {
      T best = (T)-1;
      int bi = r;
      for (int i = j + lane; i < r; i += 32) {
        T v = fabs(LU[i * ldl + j]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(FULL, best, o);
        int oi = __shfl_xor_sync(FULL, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (bi >= r) {  // NaN column: keep the diagonal, report
        bi = j;
        if (lane == 0) set_err(err, DERR_NUMERIC);
      }
      if (best == (T)0 && lane == 0) set_err(err, DERR_NUMERIC);
      if (bi != j) {
        for (int cc = lane; cc < r; cc += 32) {
          T t0 = LU[j * ldl + cc];
          LU[j * ldl + cc] = LU[bi * ldl + cc];
          LU[bi * ldl + cc] = t0;
        }
        if (lane == 0) {
          int tp = spiv[j];
          spiv[j] = spiv[bi];
          spiv[bi] = tp;
        }
      }
      __syncwarp();
      const T d = LU[j * ldl + j];
      for (int i = j + 1 + lane; i < r; i += 32) LU[i * ldl + j] /= d;
    }
    __syncthreads();
    for (int i = j + 1 + warp; i < r; i += NT / 32) {
      const T l = LU[i * ldl + j];
      for (int cc = j + 1 + lane; cc < r; cc += 32) LU[i * ldl + cc] = LU[i * ldl + cc] - l * LU[j * ldl + cc];
    }
    __syncthreads();
  }
  for (int i = tid; i < r; i += NT) spinv[spiv[i]] = i;
  for (int e = tid; e < r * r; e += NT) {
    int qi, ri;
    fdr.divmod(e, qi, ri);
    fb.LU[e] = LU[qi * ldl + ri];
  }
  for (int i = tid; i < r; i += NT) fb.piv[i] = spiv[i];
  __syncthreads();
  // X_RR^{-1} = U^{-1} L^{-1} P: column cc is U^{-1} L^{-1} e_{pinv[cc]}
  // (four partial sums per dot product to shorten the dependence chains;
  // one thread per column measured faster than the whole CTA taking a
  // rank-1 update per row step)
  for (int cc = tid; cc < r; cc += NT) {
    T *x = Xi + (size_t)cc * ldx;
    const int i0 = spinv[cc];
    for (int i = 0; i < r; i++) {
      const T *Li = LU + i * ldl;
      T s0 = (T)0, s1 = (T)0, s2 = (T)0, s3 = (T)0;
      int l = i0;  // x[l] = 0 for l < i0
      for (; l + 3 < i; l += 4) {
        s0 += Li[l] * x[l];
        s1 += Li[l + 1] * x[l + 1];
        s2 += Li[l + 2] * x[l + 2];
        s3 += Li[l + 3] * x[l + 3];
      }
      for (; l < i; l++) s0 += Li[l] * x[l];
      x[i] = (i == i0 ? (T)1 : (T)0) - ((s0 + s1) + (s2 + s3));
    }
    for (int i = r - 1; i >= 0; i--) {
      const T *Ui = LU + i * ldl;
      T s0 = (T)0, s1 = (T)0, s2 = (T)0, s3 = (T)0;
      int l = i + 1;
      for (; l + 3 < r; l += 4) {
        s0 += Ui[l] * x[l];
        s1 += Ui[l + 1] * x[l + 1];
        s2 += Ui[l + 2] * x[l + 2];
        s3 += Ui[l + 3] * x[l + 3];
      }
      for (; l < r; l++) s0 += Ui[l] * x[l];
      x[i] = (x[i] - ((s0 + s1) + (s2 + s3))) / Ui[i];
    }
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += NT) {
    int qi, ri;
    fdr.divmod(e, qi, ri);
    fb.Xi[e] = Xi[ri + (size_t)qi * ldx];
  }
  }  // cta == 0
  T *Xrj_out = scratch + (int64_t)q * sstride + (int64_t)nj * r;  // r x nj, for the Schur update
  for (int a0 = cta * CH; a0 < nj; a0 += C * CH) {
    const int na = min(CH, nj - a0);
    // raw rows A(J_a, B) and columns A(B, J_a) of the chunk (S rows come from
    // X_SR / X_RS); the row / column bases of the chunk are resolved first so
    // the element loads below are independent of one another
    if (tid < na) {
      // (code, local index) of J entry a, as in the J lists above
      const int a = a0 + tid;
      int code, la;
      if (a < k) {
        code = center;
        la = sloc[a];
      } else {
        int q2 = 0;
        while (s_nstart[q2 + 1] <= a) q2++;
        code = s_ncode[q2];
        la = lv.act_idx[s_nact[q2] + (a - s_nstart[q2])];
      }
      s_rb[tid] = s_off_in[code] + la;
      s_rl[tid] = s_ld_in[code];
      s_cb[tid] = s_off_out[code] + (int64_t)la * b;
    }
    __syncthreads();
    const FastDiv fdna(max(na, 1));
    for (int e0 = tid; e0 < na * b; e0 += 4 * NT) {
      T val[4];
      int dst[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int e = e0 + u * NT;
        val[u] = (T)0;
        dst[u] = -1;
        if (e < na * b) {
          int al, pp;
          fdna.divmod(e, pp, al);
          const int a = a0 + al;
          dst[u] = al + pp * (CH + 1);
          if (a < k) val[u] = pp >= k ? XSR[a + (pp - k) * k] : (T)0;
          else val[u] = lv.pool[s_rb[al] + (int64_t)sloc[pp] * s_rl[al]];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; u++)
        if (dst[u] >= 0) rawJ[dst[u]] = val[u];
    }
    for (int e0 = tid; e0 < na * b; e0 += 4 * NT) {
      T val[4];
      int dst[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int e = e0 + u * NT;
        val[u] = (T)0;
        dst[u] = -1;
        if (e < na * b) {
          int pp, al;
          fdb.divmod(e, al, pp);
          const int a = a0 + al;
          dst[u] = pp + al * ldb;
          if (a < k) val[u] = pp >= k ? XRS[(pp - k) + a * r] : (T)0;
          else val[u] = lv.pool[s_cb[al] + sloc[pp]];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; u++)
        if (dst[u] >= 0) rawC[dst[u]] = val[u];
    }
    __syncthreads();
    // in place: X_JR = A_JR - A_JS T (rows a >= k);  X_RJ = A_RJ - T^T A_SJ
    {
      const int ldj = CH + 1;
      T *rJ = rawJ;
      T *rC = rawC;
      const int kk = k, aa0 = a0;
      smem_gemm<T, 1>(na, r, k, rawJ, 1, ldj, Ts, k, [&](int al, int ri, T v) {
        if (aa0 + al >= kk) rJ[al + (kk + ri) * ldj] -= v;
      });
      smem_gemm<T, 2>(r, na, k, Ts, k, 1, rawC, ldb, [&](int ri, int al, T v) {
        if (aa0 + al >= kk) rC[(kk + ri) + al * ldb] -= v;
      });
    }
    __syncthreads();
    for (int e = tid; e < na * r; e += NT) {
      int ri, al;
      fdr.divmod(e, al, ri);
      Xrj_out[ri + (int64_t)(a0 + al) * r] = rawC[(k + ri) + al * ldb];
    }
    if (split) {
      // X_JR chunk to the scratch (nj x r, ld nj); E and G follow in k_elim_gemm
      T *Xjr = scratch + (int64_t)q * sstride;
      for (int e = tid; e < na * r; e += NT) {
        int al, ri;
        fdna.divmod(e, ri, al);
        Xjr[(a0 + al) + (int64_t)ri * nj] = rawJ[al + (k + ri) * (CH + 1)];
      }
      __syncthreads();
      continue;
    }
    // E chunk = X_JR chunk * X_RR^{-1};  G chunk = X_RR^{-1} * X_RJ chunk
    {
      T *Eo = fb.E, *Go = fb.G;
      const int njj = nj, rr = r, aa0 = a0;
      smem_gemm<T, 1>(na, r, r, rawJ + (size_t)k * (CH + 1), 1, CH + 1, Xi, ldx, [&](int al, int ri, T v) {
        Eo[(aa0 + al) + (int64_t)ri * njj] = v;
      });
      if (Go)  // uniform over the CTA; symmetric storage keeps no G
        smem_gemm<T, 1>(r, na, r, Xi, 1, ldx, rawC + k, ldb, [&](int ri, int al, T v) {
          Go[ri + (int64_t)(aa0 + al) * rr] = v;
        });
    }
    __syncthreads();
  }
  // the box's active DOFs are now its skeleton, kept in ascending order
  if (cta != 0) return;
  const int64_t coff = lv.cell_dof_off[c];
  for (int s1 = tid; s1 < k; s1 += NT) {
    int v = sloc[s1], rank = 0;
    for (int s2 = 0; s2 < k; s2++) rank += sloc[s2] < v;
    lv.act_idx[coff + rank] = v;
  }
  if (tid == 0) lv.act_cnt[c] = k;
}

template <typename T> int64_t elim_smem_bytes(int b, int k, int r) {
  return (int64_t)k * r * sizeof(T) + (int64_t)r * (r + 1) * sizeof(T) + (int64_t)(b + r) * sizeof(int) + 16;
}
template int64_t elim_smem_bytes<float>(int, int, int);
template int64_t elim_smem_bytes<double>(int, int, int);

// Elements of T the large-box elimination needs per box beyond X_JR / X_RJ.
// k_elim's LU (r x (r+1)) and pivots, or k_elim_lu's X_RR (r x r), r <= bmax
template <typename T> int64_t elim_ws_elems(int bmax) {
  return (int64_t)bmax * (bmax + 1) + (int64_t)bmax + 64;
}
template int64_t elim_ws_elems<float>(int);
template int64_t elim_ws_elems<double>(int);

// E = X_JR X_RR^{-1} (nj x r) and G = X_RR^{-1} X_RJ (r x nj) for the boxes
// of a phase eliminated by k_elim: blockIdx.x = box of the phase,
// blockIdx.y = a 64 x 64 output tile of E (the first tiles_e) or of G.
// X_JR (ld nj) and X_RJ (ld r) are in the box's scratch, X_RR^{-1} in the
// factor (r x r, column-major).  Shared-memory tiles of 16 along the inner
// dimension; each thread accumulates a 4 x 4 block.
template <typename T>
__global__ void __launch_bounds__(NT) k_elim_gemm(const FBox<T> *boxes, const int *box_list, const T *scratch,
                                                  int64_t sstride, int tiles_e, int tcols_e, int tcols_g) {
  __shared__ T As[16][64 + 1];
  __shared__ T Bs[16][64 + 1];
  const FBox<T> &fb = boxes[box_list[blockIdx.x]];
  const int r = fb.r, nj = fb.nj;
  if (r == 0) return;
  const T *Xjr = scratch + (int64_t)blockIdx.x * sstride;
  const T *Xrj = Xjr + (int64_t)nj * r;
  const T *Xi = fb.Xi;
  // C(i, j) = sum_l A(i, l) B(l, j); all operands column-major
  int m, n, t = blockIdx.y, tcols = tcols_e;
  const T *A, *B;
  int64_t lda, ldb, ldc;
  T *Cp;
  if (t < tiles_e) {  // E = X_JR Xi: m = nj, n = r
    m = nj, n = r, A = Xjr, lda = nj, B = Xi, ldb = r, Cp = fb.E, ldc = nj;
  } else {            // G = Xi X_RJ: m = r, n = nj
    t -= tiles_e;
    tcols = tcols_g;
    m = r, n = nj, A = Xi, lda = r, B = Xrj, ldb = r, Cp = fb.G, ldc = r;
    if (!Cp) return;  // symmetric storage keeps no G
  }
  const int i0 = (t / tcols) * 64, j0 = (t % tcols) * 64;
  if (i0 >= m || j0 >= n) return;
  const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; x++)
#pragma unroll
    for (int y = 0; y < 4; y++) acc[x][y] = (T)0;
  for (int l0 = 0; l0 < r; l0 += 16) {
    for (int e = tid; e < 16 * 64; e += NT) {
      const int ii = e % 64, ll = e / 64;  // A: consecutive rows
      As[ll][ii] = (i0 + ii < m && l0 + ll < r) ? A[(i0 + ii) + (int64_t)(l0 + ll) * lda] : (T)0;
      const int l2 = e % 16, jj = e / 16;  // B: consecutive inner index
      Bs[l2][jj] = (l0 + l2 < r && j0 + jj < n) ? B[(l0 + l2) + (int64_t)(j0 + jj) * ldb] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; u++) {
      T av[4], bv[4];
#pragma unroll
      for (int x = 0; x < 4; x++) av[x] = As[u][ti + 16 * x];
#pragma unroll
      for (int y = 0; y < 4; y++) bv[y] = Bs[u][tj + 16 * y];
#pragma unroll
      for (int x = 0; x < 4; x++)
#pragma unroll
        for (int y = 0; y < 4; y++) acc[x][y] += av[x] * bv[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < 4; y++) {
    const int j = j0 + tj + 16 * y;
    if (j >= n) continue;
#pragma unroll
    for (int x = 0; x < 4; x++) {
      const int i = i0 + ti + 16 * x;
      if (i < m) Cp[i + (int64_t)j * ldc] = acc[x][y];
    }
  }
}

// X_RR = A_RR - T^T A_SR - X_RS T (Sec. 3.1) for the boxes of a phase whose
// elimination runs in k_elim_lu, one 64 x 64 tile of X_RR per CTA: a GEMM of
// inner dimension 2k with A' = [T^T | X_RS] (r x 2k) and B' = [A_SR ; T]
// (2k x r), subtracted from A_RR.  X_RS is the first k columns of X_RJ in the
// box's scratch (formed by k_elim); X_RR goes to the box's workspace,
// column-major with leading dimension r.
template <typename T>
__global__ void __launch_bounds__(NT) k_elim_xrr(LevelDev<T> lv, const FBox<T> *boxes, const int *box_list,
                                                 T *scratch, int64_t sstride, int64_t ws_off, int tcols) {
  __shared__ T As[16][64 + 1];
  __shared__ T Bs[16][64 + 1];
  const int q = blockIdx.x;
  const FBox<T> &fb = boxes[box_list[q]];
  const int r = fb.r, k = fb.k, b = fb.b, nj = fb.nj;
  const int i0 = (blockIdx.y / tcols) * 64, j0 = (blockIdx.y % tcols) * 64;
  if (r == 0 || i0 >= r || j0 >= r) return;
  const T *Xrj = scratch + (int64_t)q * sstride + (int64_t)nj * r;
  T *M = scratch + (int64_t)q * sstride + ws_off;
  const int center = code5(0, 0, 0, lv.dim);
  const int self = lv.cell_nbr[(int64_t)fb.cell * lv.NB + center];
  const T *Aii = lv.pool + lv.pair_off[(int64_t)self * lv.NB + center];  // block (c, c), ld b
  const int *loc = fb.loc;
  const T *Tm = fb.Tm;
  const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; x++)
#pragma unroll
    for (int y = 0; y < 4; y++) acc[x][y] = (T)0;
  for (int l0 = 0; l0 < 2 * k; l0 += 16) {
    for (int e = tid; e < 16 * 64; e += NT) {
      {
        const int ii = e % 64, l = l0 + e / 64, ri = i0 + ii;
        T av = (T)0;
        if (ri < r && l < 2 * k) av = l < k ? Tm[l + (int64_t)ri * k] : Xrj[ri + (int64_t)(l - k) * r];
        As[e / 64][ii] = av;
      }
      {
        const int l2 = e % 16, jj = e / 16, l = l0 + l2, rj = j0 + jj;
        T bv = (T)0;
        if (rj < r && l < 2 * k)
          bv = l < k ? Aii[loc[l] + (int64_t)loc[k + rj] * b] : Tm[(l - k) + (int64_t)rj * k];
        Bs[l2][jj] = bv;
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; u++) {
      T av[4], bv[4];
#pragma unroll
      for (int x = 0; x < 4; x++) av[x] = As[u][ti + 16 * x];
#pragma unroll
      for (int y = 0; y < 4; y++) bv[y] = Bs[u][tj + 16 * y];
#pragma unroll
      for (int x = 0; x < 4; x++)
#pragma unroll
        for (int y = 0; y < 4; y++) acc[x][y] += av[x] * bv[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < 4; y++) {
    const int rj = j0 + tj + 16 * y;
    if (rj >= r) continue;
#pragma unroll
    for (int x = 0; x < 4; x++) {
      const int ri = i0 + ti + 16 * x;
      if (ri < r) M[ri + (int64_t)rj * r] = Aii[loc[k + ri] + (int64_t)loc[k + rj] * b] - acc[x][y];
    }
  }
}

// (value, index) argmax over a warp: largest value, ties to the lowest index
template <typename T> __device__ __forceinline__ void warp_argmax(T &best, int &bi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T ov = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
}

constexpr int NLU = 1024;  // threads of k_elim_lu

template <typename T> size_t elim_lu_smem(int r, int nbp) {
  return 2 * (size_t)nbp * r * sizeof(T) + (size_t)r * sizeof(int) + 16;
}

// LU with partial pivoting of X_RR (largest |entry|, ties to the lowest row;
// X_RR = P^T L U), X_RR^{-1} = U^{-1} L^{-1} P and the box's skeleton list,
// one CTA of 1024 threads per box, for boxes too wide for k_elim's
// shared-memory form.  Blocked right-looking LU with panels of NBP columns:
// the panel is factored in shared memory (a block-wide argmax per column),
// its row interchanges are applied to the other columns, U12 = L11^{-1} A12
// by one thread per column, and A22 -= L21 U12 with each lane accumulating a
// 4 x 4 block.  X_RR^{-1} by blocked forward and back substitution on the
// columns of the identity, NBP rows at a time, the block rows of L and U
// staged in shared memory.  X_RR (column-major, ld r) is in the workspace.
template <typename T, int NBP>
__global__ void __launch_bounds__(NLU) k_elim_lu(LevelDev<T> lv, FBox<T> *boxes, const int *box_list, T *scratch,
                                                 int64_t sstride, int64_t ws_off, int *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T s_bv[32];
  __shared__ int s_bi[32], s_p, s_swp[NBP];
  FBox<T> &fb = boxes[box_list[blockIdx.x]];
  const int r = fb.r, k = fb.k, c = fb.cell;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T *M = scratch + (int64_t)blockIdx.x * sstride + ws_off;
  T *P = reinterpret_cast<T *>(smem_raw);  // panel: P[jj * r + i], rows i in [j0, r)
  T *U = P + (int64_t)NBP * r;              // U12: U[t * r + column]
  int *perm = reinterpret_cast<int *>(U + (int64_t)NBP * r);
  if (r > 0) {
    for (int i = tid; i < r; i += NLU) perm[i] = i;
    for (int j0 = 0; j0 < r; j0 += NBP) {
      const int nb = min(NBP, r - j0), h = r - j0;
      for (int e = tid; e < nb * h; e += NLU) {
        const int jj = e / h, i = j0 + e % h;
        P[jj * r + i] = M[i + (int64_t)(j0 + jj) * r];
      }
      __syncthreads();
      for (int jj = 0; jj < nb; jj++) {
        const int j = j0 + jj;
        T best = (T)-1;
        int bi = r;
        for (int i = j + tid; i < r; i += NLU) {
          const T v = fabs(P[jj * r + i]);
          if (v > best) {
            best = v;
            bi = i;
          }
        }
        warp_argmax(best, bi);
        if (lane == 0) {
          s_bv[warp] = best;
          s_bi[warp] = bi;
        }
        __syncthreads();
        if (warp == 0) {
          best = s_bv[lane];
          bi = s_bi[lane];
          warp_argmax(best, bi);
          if (lane == 0) {
            if (bi >= r) {  // NaN column: keep the diagonal, report
              bi = j;
              set_err(err, DERR_NUMERIC);
            }
            if (best == (T)0) set_err(err, DERR_NUMERIC);
            s_p = bi;
            s_swp[jj] = bi;
          }
        }
        __syncthreads();
        const int p = s_p;
        if (p != j) {
          if (tid < nb) {
            const T t0 = P[tid * r + j];
            P[tid * r + j] = P[tid * r + p];
            P[tid * r + p] = t0;
          }
          if (tid == NLU - 1) {
            const int tp = perm[j];
            perm[j] = perm[p];
            perm[p] = tp;
          }
          __syncthreads();
        }
        const T d = P[jj * r + j];
        for (int i = j + 1 + tid; i < r; i += NLU) P[jj * r + i] /= d;
        __syncthreads();
        const int rows = r - j - 1, cols = nb - jj - 1;
        for (int e = tid; e < rows * cols; e += NLU) {
          const int i = j + 1 + e % rows, cc = jj + 1 + e / rows;
          P[cc * r + i] -= P[jj * r + i] * P[cc * r + j];
        }
        __syncthreads();
      }
      for (int e = tid; e < nb * h; e += NLU) {
        const int jj = e / h, i = j0 + e % h;
        M[i + (int64_t)(j0 + jj) * r] = P[jj * r + i];
      }
      // the panel's row interchanges, in order, on the columns outside it
      for (int cc = tid; cc < r; cc += NLU) {
        if (cc >= j0 && cc < j0 + nb) continue;
        T *col = M + (int64_t)cc * r;
        for (int jj = 0; jj < nb; jj++) {
          const int p = s_swp[jj], j = j0 + jj;
          if (p != j) {
            const T t0 = col[j];
            col[j] = col[p];
            col[p] = t0;
          }
        }
      }
      __syncthreads();
      const int c0 = j0 + nb, nc = r - c0;
      if (nc > 0) {
        // U12 = L11^{-1} A12, one thread per column right of the panel
        for (int cc = c0 + tid; cc < r; cc += NLU) {
          T u[NBP];
          T *col = M + (int64_t)cc * r + j0;
#pragma unroll
          for (int t = 0; t < NBP; t++) u[t] = t < nb ? col[t] : (T)0;
#pragma unroll
          for (int t = 1; t < NBP; t++)
            if (t < nb) {
              T a = u[t];
#pragma unroll
              for (int t2 = 0; t2 < t; t2++) a -= P[t2 * r + j0 + t] * u[t2];
              u[t] = a;
            }
#pragma unroll
          for (int t = 0; t < NBP; t++)
            if (t < nb) {
              col[t] = u[t];
              U[t * r + cc] = u[t];
            }
        }
        __syncthreads();
        // A22 -= L21 U12: a warp takes 128 rows x 4 columns, a lane rows
        // lane + 32x (x < 4) of them
        const int ublk = (nc + 127) / 128, cblk = (nc + 3) / 4;
        for (int w = warp; w < ublk * cblk; w += NLU / 32) {
          const int ib = c0 + (w % ublk) * 128 + lane, cb = c0 + (w / ublk) * 4;
          T acc[4][4];
#pragma unroll
          for (int x = 0; x < 4; x++)
#pragma unroll
            for (int y = 0; y < 4; y++) acc[x][y] = (T)0;
          for (int t = 0; t < nb; t++) {
            T lv4[4], uv[4];
#pragma unroll
            for (int x = 0; x < 4; x++) lv4[x] = ib + 32 * x < r ? P[t * r + ib + 32 * x] : (T)0;
#pragma unroll
            for (int y = 0; y < 4; y++) uv[y] = cb + y < r ? U[t * r + cb + y] : (T)0;
#pragma unroll
            for (int x = 0; x < 4; x++)
#pragma unroll
              for (int y = 0; y < 4; y++) acc[x][y] += lv4[x] * uv[y];
          }
#pragma unroll
          for (int y = 0; y < 4; y++) {
            if (cb + y >= r) continue;
#pragma unroll
            for (int x = 0; x < 4; x++)
              if (ib + 32 * x < r) M[ib + 32 * x + (int64_t)(cb + y) * r] -= acc[x][y];
          }
        }
      }
      __syncthreads();
    }
    // the factors, row-major as the sweeps read them
    for (int e = tid; e < r * r; e += NLU) fb.LU[e] = M[e / r + (int64_t)(e % r) * r];
    for (int i = tid; i < r; i += NLU) fb.piv[i] = perm[i];
    // X_RR^{-1} = U^{-1} L^{-1} P: column perm[i] of it is U^{-1} L^{-1} e_i.
    // Forward: w = L^{-1} e_i, NBP rows at a time, rows m0.. of L in P
    T *Xi = fb.Xi;
    for (int m0 = 0; m0 < r; m0 += NBP) {
      const int nb = min(NBP, r - m0);
      for (int e = tid; e < NBP * (m0 + nb); e += NLU) {
        const int t = e % NBP, l = e / NBP;
        P[t + l * NBP] = t < nb ? M[m0 + t + (int64_t)l * r] : (T)0;
      }
      __syncthreads();
      for (int i = tid; i < r; i += NLU) {
        T *w = Xi + (int64_t)perm[i] * r;
        T acc[NBP];
#pragma unroll
        for (int t = 0; t < NBP; t++) acc[t] = m0 + t == i ? (T)1 : (T)0;
        // from the warp's first column on (w[l] = 0 for l < i): the same l
        // in every lane, so the reads of P are broadcasts
        for (int l = i - lane; l < m0; l++) {
          const T wl = w[l];
#pragma unroll
          for (int t = 0; t < NBP; t++) acc[t] -= P[t + l * NBP] * wl;
        }
#pragma unroll
        for (int t = 1; t < NBP; t++)
          if (t < nb) {
            T a = acc[t];
#pragma unroll
            for (int t2 = 0; t2 < t; t2++) a -= P[t + (m0 + t2) * NBP] * acc[t2];
            acc[t] = a;
          }
#pragma unroll
        for (int t = 0; t < NBP; t++)
          if (t < nb) w[m0 + t] = m0 + t < i ? (T)0 : acc[t];
      }
      __syncthreads();
    }
    // Back: z = U^{-1} w, from the last block of rows up
    for (int m0 = ((r - 1) / NBP) * NBP; m0 >= 0; m0 -= NBP) {
      const int nb = min(NBP, r - m0);
      for (int e = tid; e < NBP * (r - m0); e += NLU) {
        const int t = e % NBP, l = m0 + e / NBP;
        P[t + (l - m0) * NBP] = t < nb ? M[m0 + t + (int64_t)l * r] : (T)0;
      }
      __syncthreads();
      for (int i = tid; i < r; i += NLU) {
        T *w = Xi + (int64_t)perm[i] * r;
        T acc[NBP];
#pragma unroll
        for (int t = 0; t < NBP; t++) acc[t] = t < nb ? w[m0 + t] : (T)0;
        for (int l = m0 + nb; l < r; l++) {
          const T zl = w[l];
#pragma unroll
          for (int t = 0; t < NBP; t++) acc[t] -= P[t + (l - m0) * NBP] * zl;
        }
#pragma unroll
        for (int t = NBP - 1; t >= 0; t--) {
          if (t >= nb) continue;
          T a = acc[t];
#pragma unroll
          for (int t2 = t + 1; t2 < NBP; t2++)
            if (t2 < nb) a -= P[t + t2 * NBP] * acc[t2];
          acc[t] = a / P[t + t * NBP];
        }
#pragma unroll
        for (int t = 0; t < NBP; t++)
          if (t < nb) w[m0 + t] = acc[t];
      }
      __syncthreads();
    }
  }
  // the box's active DOFs are now its skeleton, kept in ascending order
  const int64_t coff = lv.cell_dof_off[c];
  for (int s = tid; s < k; s += NLU) {
    const int v = fb.loc[s];
    int rank = 0;
    for (int s2 = 0; s2 < k; s2++) rank += fb.loc[s2] < v;
    lv.act_idx[coff + rank] = v;
  }
  if (tid == 0) lv.act_cnt[c] = k;
}

// Shape of the next k_elim2 launch on this thread: (split << 4) | CTAs per
// box, or 0 for the built-in choice.  Set by the host's autotuner.
static thread_local int elim_shape_hint = 0;
void set_elim_shape(int h) { elim_shape_hint = h; }

template <typename T>
void launch_elim(const LevelDev<T> &lv, FBox<T> *boxes, const int *box_list, int nbox, int bmax, T *scratch,
                 int64_t scratch_stride, const Overflow<T> &ovf, cudaStream_t st, int *err, int njmax) {
  if (nbox == 0) return;
  const bool force_general = bmax < 0;  // large-box path requested
  if (force_general) bmax = -bmax;
  // Built in: phases of fewer than 300 boxes (upper levels) leave X_JR and
  // X_RJ in the scratch and form E and G in k_elim_gemm, spread over the
  // whole GPU; large phases form them in the one-CTA-per-box kernel
  // (measured on the 512^2 grid).  The autotuner may choose otherwise.
  int split = nbox < 300 ? 1 : 0;
  int C = split ? std::min(8, std::max(1, (300 + nbox - 1) / nbox)) : 1;  // CTAs per box
  if (elim_shape_hint > 0) {
    split = (elim_shape_hint >> 4) & 1;
    C = split ? std::max(1, elim_shape_hint & 15) : 1;
  }
  const int tr = (bmax + 63) / 64, tn = (std::max(njmax, 1) + 63) / 64;
  if (!force_general) {
    // worst case over k + r = b of the shared-memory form
    size_t worst = 0;
    for (int r = 0; r <= bmax; r++) worst = std::max(worst, elim2_smem<T>(bmax, bmax - r, r));
    // boxes of up to 128 DOFs (wider ones take the blocked LU below)
    if (worst <= (size_t)(220 << 10) && bmax <= 128) {
      cudaFuncSetAttribute(k_elim2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)worst);
      k_elim2<T><<<nbox * C, NT, worst, st>>>(lv, boxes, box_list, scratch, scratch_stride, ovf, err, split, C);
      count_launch();
      if (split) {
        k_elim_gemm<T><<<dim3(nbox, 2 * tn * tr), NT, 0, st>>>(boxes, box_list, scratch, scratch_stride, tn * tr, tr,
                                                                 tn);
        count_launch();
      }
      return;
    }
  }
  // the global workspace sits after the X_JR / X_RJ scratch of the box
  const int64_t ws_off = scratch_stride - elim_ws_elems<T>(bmax);
  const int tiles_e = tn * tr;  // E: nj x r
  const int tiles_g = tr * tn;  // G: r x nj
  if (!force_general) {
    // boxes wider than k_elim2 takes: X_JR and X_RJ over up to 64 CTAs per
    // box, X_RR as tiles, the LU and X_RR^{-1} blocked in one 1024-thread CTA
    // per box (3D 32^3 grid: 83 -> 26 ms at eps 1e-3, b ~ 200, and
    // 1063 -> 152 ms at eps 1e-6, b = 448, against k_elim)
    int nbp = sizeof(T) == 4 ? 32 : 16;
    while (nbp > 8 && elim_lu_smem<T>(bmax, nbp) > (size_t)(220 << 10)) nbp /= 2;
    const size_t lsm = elim_lu_smem<T>(bmax, nbp);
    if (lsm <= (size_t)(220 << 10)) {
      const int Cb = std::min(64, std::max(1, (1216 + nbox - 1) / nbox));
      k_elim<T><<<nbox * Cb, NT, 0, st>>>(lv, boxes, box_list, scratch, scratch_stride, ws_off, ovf, err, Cb, 1);
      k_elim_xrr<T><<<dim3(nbox, tr * tr), NT, 0, st>>>(lv, boxes, box_list, scratch, scratch_stride, ws_off, tr);
      if (nbp == 8) {
        cudaFuncSetAttribute(k_elim_lu<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm);
        k_elim_lu<T, 8><<<nbox, NLU, lsm, st>>>(lv, boxes, box_list, scratch, scratch_stride, ws_off, err);
      } else if (nbp == 16) {
        cudaFuncSetAttribute(k_elim_lu<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm);
        k_elim_lu<T, 16><<<nbox, NLU, lsm, st>>>(lv, boxes, box_list, scratch, scratch_stride, ws_off, err);
      } else {
        cudaFuncSetAttribute(k_elim_lu<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm);
        k_elim_lu<T, 32><<<nbox, NLU, lsm, st>>>(lv, boxes, box_list, scratch, scratch_stride, ws_off, err);
      }
      k_elim_gemm<T><<<dim3(nbox, tiles_e + tiles_g), NT, 0, st>>>(boxes, box_list, scratch, scratch_stride,
                                                                    tiles_e, tr, tn);
      count_launch(4);
      return;
    }
  }
  // one CTA per box, everything in k_elim (the forced large-box path, kept
  // as the plain form the other paths are checked against, and boxes too
  // wide for k_elim_lu's shared memory)
  const int Cg = force_general ? 1 : std::min(8, std::max(1, (300 + nbox - 1) / nbox));
  k_elim<T><<<nbox * Cg, NT, 0, st>>>(lv, boxes, box_list, scratch, scratch_stride, ws_off, ovf, err, Cg, 0);
  // E and G: tiles of 64 x 64 over nj x r (E) and r x nj (G), nj <= njmax, r <= bmax
  k_elim_gemm<T><<<dim3(nbox, tiles_e + tiles_g), NT, 0, st>>>(boxes, box_list, scratch, scratch_stride, tiles_e,
                                                              tr, tn);
  count_launch(2);
}

// ---------------------------------------------------------------------------
// Schur complement update X_JJ -= E G, scattered into the pair blocks
// ---------------------------------------------------------------------------

constexpr int ST = 64;   // output tile
constexpr int SK = 16;   // inner chunk

// S_JJ = X_JJ - X_JR X_RR^{-1} X_RJ = X_JJ - E X_RJ (Sec. 2.1); X_RJ is still in
// the elimination scratch of this phase (r x nj column-major after X_JR).
template <typename T>
__global__ void __launch_bounds__(NT) k_schur(LevelDev<T> lv, const FBox<T> *boxes, const int *box_list,
                                              int tiles1, const T *scratch, int64_t sstride) {
  __shared__ T Es[SK][ST + 1];
  __shared__ T Gs[SK][ST + 1];
  __shared__ int s_cell3[27];
  // scatter tables of the tile: 3^d code and local index of its rows and
  // columns of J, the pool offset of the pair block (row cell, column cell)
  // for every pair of codes, and the leading dimension of each row cell
  __shared__ int s_rc[ST], s_rl[ST], s_cc[ST], s_cl[ST], s_ld[27];
  __shared__ int64_t s_po[27 * 27];
  const int bi = blockIdx.x / (tiles1 * tiles1);
  const int tt = blockIdx.x % (tiles1 * tiles1);
  const FBox<T> &fb = boxes[box_list[bi]];
  const int nj = fb.nj, r = fb.r, dim = lv.dim;
  const int a0 = (tt / tiles1) * ST, c0 = (tt % tiles1) * ST;
  if (a0 >= nj || c0 >= nj || r == 0) return;
  const T *Xrj = scratch + (int64_t)bi * sstride + (int64_t)nj * r;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int nc3 = dim == 3 ? 27 : 9;
  if (tid < nc3) {
    int dx, dy, dz;
    decode3(tid, dim, dx, dy, dz);
    const int cl = lv.cell_nbr[(int64_t)fb.cell * lv.NB + code5(dx, dy, dz, dim)];
    s_cell3[tid] = cl;
    s_ld[tid] = cl >= 0 ? lv.cell_b[cl] : 0;
  }
  if (tid < ST) {
    const int a = a0 + tid, cc = c0 + tid;
    s_rc[tid] = a < nj ? fb.Jnb[a] : 0;
    s_rl[tid] = a < nj ? fb.Jloc[a] : 0;
    s_cc[tid] = cc < nj ? fb.Jnb[cc] : 0;
    s_cl[tid] = cc < nj ? fb.Jloc[cc] : 0;
  }
  __syncthreads();
  for (int e = tid; e < nc3 * nc3; e += NT) {
    const int ra = e / nc3, rc = e % nc3;
    const int ca = s_cell3[ra];
    int adx, ady, adz, cdx, cdy, cdz;
    decode3(ra, dim, adx, ady, adz);
    decode3(rc, dim, cdx, cdy, cdz);
    s_po[e] = ca >= 0 ? lv.pair_off[(int64_t)ca * lv.NB + code5(cdx - adx, cdy - ady, cdz - adz, dim)] : -1;
  }
  T acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; x++)
#pragma unroll
    for (int y = 0; y < 4; y++) acc[x][y] = (T)0;
  for (int r0 = 0; r0 < r; r0 += SK) {
    for (int e = tid; e < SK * ST; e += NT) {
      int u = e / ST, i = e % ST;
      int ri = r0 + u;
      Es[u][i] = (ri < r && a0 + i < nj) ? fb.E[(a0 + i) + (int64_t)ri * nj] : (T)0;
      int u2 = e % SK, i2 = e / SK;
      int ri2 = r0 + u2;
      Gs[u2][i2] = (ri2 < r && c0 + i2 < nj) ? Xrj[ri2 + (int64_t)(c0 + i2) * r] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < SK; u++) {
      T ev[4], gv[4];
#pragma unroll
      for (int x = 0; x < 4; x++) ev[x] = Es[u][tx + 16 * x];
#pragma unroll
      for (int y = 0; y < 4; y++) gv[y] = Gs[u][ty + 16 * y];
#pragma unroll
      for (int x = 0; x < 4; x++)
#pragma unroll
        for (int y = 0; y < 4; y++) acc[x][y] += ev[x] * gv[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < 4; y++) {
    const int jc = ty + 16 * y;
    if (c0 + jc >= nj) continue;
    const int codec = s_cc[jc], lc = s_cl[jc];
#pragma unroll
    for (int x = 0; x < 4; x++) {
      const int ia = tx + 16 * x;
      if (a0 + ia >= nj) continue;
      const int codea = s_rc[ia];
      const int64_t off = s_po[codea * nc3 + codec];
      T *dst = lv.pool + off + s_rl[ia] + (int64_t)lc * s_ld[codea];
      if (lv.shared) atomicAdd(dst, -acc[x][y]);  // pair blocks other boxes of the phase update too
      else *dst -= acc[x][y];
    }
  }
}

template <typename T>
void launch_schur(const LevelDev<T> &lv, const FBox<T> *boxes, const int *box_list, int nbox, int njmax,
                  const T *scratch, int64_t scratch_stride, cudaStream_t st) {
  if (nbox == 0) return;
  int tiles1 = (njmax + ST - 1) / ST;
  int64_t grid = (int64_t)nbox * tiles1 * tiles1;
  k_schur<T><<<(unsigned)grid, NT, 0, st>>>(lv, boxes, box_list, tiles1, scratch, scratch_stride); count_launch();
}

// ---------------------------------------------------------------------------
// Dense LU with partial pivoting (top block), row-major, blocked
// ---------------------------------------------------------------------------

constexpr int LB = 32;

// Panel of nb <= LB columns at kb (rows kb..n-1), factored with partial
// pivoting (largest |entry|, ties to the lowest row) in a column-major copy W,
// so that the argmax, the scaling and the rank-1 updates read consecutive
// addresses; each thread loads all of a row's panel entries before it
// updates them.  The row interchanges go to swp (local rows) and to the
// permutation; k_lu_trsm applies them to the other columns.
template <typename T>
__global__ void __launch_bounds__(1024) k_lu_panel(T *A, int n, int kb, int nb, int *piv, T *Wg, int *swp,
                                                   int *err, int in_smem) {
  constexpr int CH = sizeof(T) == 4 ? 16 : 8;  // panel entries a thread holds at once
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T s_val[32];
  __shared__ int s_idx[32];
  __shared__ T s_prow[LB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x / 32;
  const int h = n - kb;  // panel rows kb..n-1; W column-major, ld h
  // the panel in shared memory when it fits, else in the global workspace
  T *W = in_smem ? reinterpret_cast<T *>(smem_raw) : Wg;
  for (int e = tid; e < h * nb; e += blockDim.x) {
    const int i = e / nb, jj = e % nb;
    W[(int64_t)jj * h + i] = A[(int64_t)(kb + i) * n + kb + jj];
  }
  __syncthreads();
  for (int jj = 0; jj < nb; jj++) {
    T *wc = W + (int64_t)jj * h;
    T best = (T)-1;
    int bi = h;
    for (int i = jj + tid; i < h; i += blockDim.x) {
      const T v = fabs(wc[i]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    warp_argmax(best, bi);
    if (lane == 0) {
      s_val[warp] = best;
      s_idx[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      best = lane < nwarp ? s_val[lane] : (T)-1;
      bi = lane < nwarp ? s_idx[lane] : h;
      warp_argmax(best, bi);
      if (lane == 0) {
        if (bi >= h) {  // NaN column: keep the diagonal, report
          bi = jj;
          set_err(err, DERR_NUMERIC);
        }
        if (best == (T)0) set_err(err, DERR_NUMERIC);
        s_idx[0] = bi;
        swp[jj] = bi;
        const int tp = piv[kb + jj];
        piv[kb + jj] = piv[kb + bi];
        piv[kb + bi] = tp;
      }
    }
    __syncthreads();
    const int p = s_idx[0];
    if (tid < nb) {  // interchange rows jj and p of the panel; keep row jj
      const T vj = W[(int64_t)tid * h + jj], vp = W[(int64_t)tid * h + p];
      if (p != jj) {
        W[(int64_t)tid * h + jj] = vp;
        W[(int64_t)tid * h + p] = vj;
      }
      s_prow[tid] = p != jj ? vp : vj;
    }
    __syncthreads();
    const T d = s_prow[jj];
    for (int i = jj + 1 + tid; i < h; i += blockDim.x) {
      const T l = wc[i] / d;
      wc[i] = l;
      T *wi = W + i;  // row i of the panel: wi[c * h], c < LB (n * LB < 2^31)
      for (int c0 = jj + 1; c0 < nb; c0 += CH) {
        T v[CH];
#pragma unroll
        for (int u = 0; u < CH; u++)
          if (c0 + u < nb) v[u] = wi[(c0 + u) * h];
#pragma unroll
        for (int u = 0; u < CH; u++)
          if (c0 + u < nb) wi[(c0 + u) * h] = v[u] - l * s_prow[c0 + u];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < h * nb; e += blockDim.x) {
    const int i = e / nb, jj = e % nb;
    A[(int64_t)(kb + i) * n + kb + jj] = W[(int64_t)jj * h + i];
  }
}

// The panel's row interchanges (swp, in order) on every column outside it,
// then U12 = L11^{-1} A12 for the columns right of it; one thread per column
template <typename T> __global__ void k_lu_trsm(T *A, int n, int kb, int nb, const int *swp) {
  const int cc = blockIdx.x * blockDim.x + threadIdx.x;
  if (cc >= n || (cc >= kb && cc < kb + nb)) return;
  for (int jj = 0; jj < nb; jj++) {
    const int p = swp[jj];
    if (p != jj) {
      const T t0 = A[(int64_t)(kb + jj) * n + cc];
      A[(int64_t)(kb + jj) * n + cc] = A[(int64_t)(kb + p) * n + cc];
      A[(int64_t)(kb + p) * n + cc] = t0;
    }
  }
  if (cc < kb) return;
  for (int i = kb; i < kb + nb; i++) {
    T s = A[(int64_t)i * n + cc];
    for (int l = kb; l < i; l++) s -= A[(int64_t)i * n + l] * A[(int64_t)l * n + cc];
    A[(int64_t)i * n + cc] = s;
  }
}

// A22 -= L21 U12 (64 x 64 tiles, inner dimension nb <= 32)
template <typename T> __global__ void __launch_bounds__(NT) k_lu_gemm(T *A, int n, int kb, int nb) {
  __shared__ T Ls[64][LB + 1];
  __shared__ T Us[LB][64 + 1];
  const int s0 = kb + nb;
  const int i0 = s0 + blockIdx.y * 64, c0 = s0 + blockIdx.x * 64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < 64 * LB; e += NT) {
    int i = e / LB, l = e % LB;
    Ls[i][l] = (i0 + i < n && l < nb) ? A[(int64_t)(i0 + i) * n + kb + l] : (T)0;
    int l2 = e / 64, c2 = e % 64;
    Us[l2][c2] = (c0 + c2 < n && l2 < nb) ? A[(int64_t)(kb + l2) * n + c0 + c2] : (T)0;
  }
  __syncthreads();
  T acc[4][4] = {};
  for (int l = 0; l < nb; l++) {
#pragma unroll
    for (int x = 0; x < 4; x++)
#pragma unroll
      for (int y = 0; y < 4; y++) acc[x][y] += Ls[ty + 16 * x][l] * Us[l][tx + 16 * y];
  }
#pragma unroll
  for (int x = 0; x < 4; x++) {
    int i = i0 + ty + 16 * x;
    if (i >= n) continue;
#pragma unroll
    for (int y = 0; y < 4; y++) {
      int cc = c0 + tx + 16 * y;
      if (cc < n) A[(int64_t)i * n + cc] -= acc[x][y];
    }
  }
}

template <typename T> __global__ void k_iota(int *p, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

template <typename T> void launch_dense_lu(T *A, int n, int *piv, T *W, cudaStream_t st, int *err) {
  if (n <= 0) return;
  k_iota<T><<<(n + 255) / 256, 256, 0, st>>>(piv, n); count_launch();
  for (int kb = 0; kb < n; kb += LB) {
    int nb = min(LB, n - kb);
    int *swp = reinterpret_cast<int *>(W + (int64_t)n * LB);
    // the panel (n - kb rows x nb) in shared memory when it fits, and then
    // a CTA of 256 threads (fewer warps at every barrier of the column steps)
    const size_t psm = (size_t)(n - kb) * nb * sizeof(T);
    const bool in_smem = psm <= (size_t)(160u << 10);
    if (in_smem) {
      if (!capturing(st))
        cudaFuncSetAttribute(k_lu_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 << 10);
      k_lu_panel<T><<<1, 256, psm, st>>>(A, n, kb, nb, piv, W, swp, err, 1);
    } else {
      k_lu_panel<T><<<1, 1024, 0, st>>>(A, n, kb, nb, piv, W, swp, err, 0);
    }
    count_launch();
    int rem = n - kb - nb;
    if (rem > 0 || kb > 0) {
      k_lu_trsm<T><<<(n + 127) / 128, 128, 0, st>>>(A, n, kb, nb, swp); count_launch();
    }
    if (rem > 0) {
      dim3 g((rem + 63) / 64, (rem + 63) / 64);
      k_lu_gemm<T><<<g, NT, 0, st>>>(A, n, kb, nb); count_launch();
    }
  }
}

// ---------------------------------------------------------------------------
// Sweeps: apply F (Eq. 3.10) or F^{-1} (Eq. 3.11) box by box
// ---------------------------------------------------------------------------

// In-place LU solve / multiply on a vector in shared memory by one warp.
template <typename T>
__device__ void warp_lu_solve(const T *LU, const int *piv, int r, T *x, T *tmp, int lane) {
  for (int i = lane; i < r; i += 32) tmp[i] = x[piv[i]];
  __syncwarp();
  for (int i = 0; i < r; i++) {
    T yi = tmp[i];
    for (int l = i + 1 + lane; l < r; l += 32) tmp[l] -= LU[(int64_t)l * r + i] * yi;
    __syncwarp();
  }
  for (int i = r - 1; i >= 0; i--) {
    T yi = tmp[i] / LU[(int64_t)i * r + i];
    __syncwarp();
    if (lane == 0) tmp[i] = yi;
    for (int l = lane; l < i; l += 32) tmp[l] -= LU[(int64_t)l * r + i] * yi;
    __syncwarp();
  }
  for (int i = lane; i < r; i += 32) x[i] = tmp[i];
  __syncwarp();
}

// G(ri, a) of a box: its stored G, or E(a, ri) under symmetric storage
// (G = E^T for the symmetric kernels, Sec. 3.3).
template <typename T> __device__ __forceinline__ T gval(const FBox<T> &fb, int ri, int a) {
  return fb.G ? __ldg(fb.G + ri + (int64_t)a * fb.r) : __ldg(fb.E + a + (int64_t)ri * fb.nj);
}

// vJ(a, c): the J entries, from the shared copy or, for boxes whose J does
// not fit in shared memory, straight from the vector
#define VJ(a, c) (jsh ? vJ[(a) * nrhs + (c)] : v[fb.J[a] * nrhs + (c)])

template <typename T>
__global__ void __launch_bounds__(NT) k_sweep(int mode, const FBox<T> *boxes, int first, T *v, int nrhs, int jsh,
                                              int shared) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FBox<T> &fb = boxes[first + blockIdx.x];
  const int k = fb.k, r = fb.r, nj = fb.nj;
  if (r == 0) return;
  const int tid = threadIdx.x;
  // vectors in shared memory, layout [i * nrhs + c]
  T *vS = reinterpret_cast<T *>(smem_raw);   // k
  T *vR = vS + (size_t)k * nrhs;              // r
  T *tmp = vR + (size_t)r * nrhs;             // r
  T *vJ = tmp + (size_t)r * nrhs;             // nj (when jsh)
  const int64_t *S = fb.ids, *Rr = fb.ids + k;
  for (int e = tid; e < k * nrhs; e += NT) vS[e] = v[S[e / nrhs] * nrhs + e % nrhs];
  for (int e = tid; e < r * nrhs; e += NT) vR[e] = v[Rr[e / nrhs] * nrhs + e % nrhs];
  if (mode == SWEEP_SOLVE_BWD && jsh)
    for (int e = tid; e < nj * nrhs; e += NT) vJ[e] = v[fb.J[e / nrhs] * nrhs + e % nrhs];
  __syncthreads();
  if (mode == SWEEP_SOLVE_FWD) {
    // U_T: v_R -= T^T v_S
    for (int e = tid; e < r * nrhs; e += NT) {
      int ri = e % r, c = e / r;
      T acc = (T)0;
      for (int q = 0; q < k; q++) acc += fb.Tm[q + (int64_t)ri * k] * vS[q * nrhs + c];
      tmp[ri * nrhs + c] = vR[ri * nrhs + c] - acc;
    }
    __syncthreads();
    // L: v_J -= E v_R
    for (int e = tid; e < nj * nrhs; e += NT) {
      int a = e % nj, c = e / nj;
      T acc = (T)0;
      for (int ri = 0; ri < r; ri++) acc += fb.E[a + (int64_t)ri * nj] * tmp[ri * nrhs + c];
      if (shared) atomicAdd(v + fb.J[a] * nrhs + c, -acc);  // near DOFs other boxes of the phase update too
      else v[fb.J[a] * nrhs + c] -= acc;
    }
    // D^{-1} on R (v_R is final for this box): x_R = X_RR^{-1} v_R
    for (int e = tid; e < r * nrhs; e += NT) {
      int i = e % r, c = e / r;
      T acc = (T)0;
      for (int l = 0; l < r; l++) acc += fb.Xi[i + (int64_t)l * r] * tmp[l * nrhs + c];
      v[Rr[i] * nrhs + c] = acc;
    }
  } else if (mode == SWEEP_SOLVE_BWD) {
    // U: v_R -= G v_J
    for (int e = tid; e < r * nrhs; e += NT) {
      int ri = e % r, c = e / r;
      T acc = (T)0;
      for (int a = 0; a < nj; a++) acc += gval(fb, ri, a) * VJ(a, c);
      vR[ri * nrhs + c] -= acc;
    }
    __syncthreads();
    // L_T: v_S -= T v_R
    for (int e = tid; e < k * nrhs; e += NT) {
      int q = e % k, c = e / k;
      T acc = (T)0;
      for (int ri = 0; ri < r; ri++) acc += fb.Tm[q + (int64_t)ri * k] * vR[ri * nrhs + c];
      v[S[q] * nrhs + c] = vS[q * nrhs + c] - acc;
    }
    for (int e = tid; e < r * nrhs; e += NT) v[Rr[e / nrhs] * nrhs + e % nrhs] = vR[e];
  } else if (mode == SWEEP_APPLY_FWD || mode == SWEEP_APPLY_W) {
    // L_T^{-1}: v_S += T v_R
    for (int e = tid; e < k * nrhs; e += NT) {
      int q = e % k, c = e / k;
      T acc = (T)0;
      for (int ri = 0; ri < r; ri++) acc += fb.Tm[q + (int64_t)ri * k] * vR[ri * nrhs + c];
      vS[q * nrhs + c] += acc;
      v[S[q] * nrhs + c] = vS[q * nrhs + c];
    }
    __syncthreads();
    // gather v_J (its S part was just updated, also in v)
    if (jsh)
      for (int e = tid; e < nj * nrhs; e += NT) {
        int a = e / nrhs, c = e % nrhs;
        vJ[e] = a < k ? vS[a * nrhs + c] : v[fb.J[a] * nrhs + c];
      }
    __syncthreads();
    // U^{-1}: v_R += G v_J
    for (int e = tid; e < r * nrhs; e += NT) {
      int ri = e % r, c = e / r;
      T acc = (T)0;
      for (int a = 0; a < nj; a++) acc += gval(fb, ri, a) * VJ(a, c);
      vR[ri * nrhs + c] += acc;
    }
    __syncthreads();
    if (mode == SWEEP_APPLY_W) {  // the W product only: v_R as it stands
      for (int e = tid; e < r * nrhs; e += NT) v[Rr[e / nrhs] * nrhs + e % nrhs] = vR[e];
      return;
    }
    // D: y_R = P^T L U v_R
    for (int e = tid; e < r * nrhs; e += NT) {
      int i = e % r, c = e / r;
      T acc = (T)0;
      for (int l = i; l < r; l++) acc += fb.LU[(int64_t)i * r + l] * vR[l * nrhs + c];
      tmp[i * nrhs + c] = acc;
    }
    __syncthreads();
    for (int e = tid; e < r * nrhs; e += NT) {
      int i = e % r, c = e / r;
      T acc = tmp[i * nrhs + c];
      for (int l = 0; l < i; l++) acc += fb.LU[(int64_t)i * r + l] * tmp[l * nrhs + c];
      v[Rr[fb.piv[i]] * nrhs + c] = acc;
    }
  } else {  // SWEEP_APPLY_BWD
    // L^{-1}: v_J += E v_R
    for (int e = tid; e < nj * nrhs; e += NT) {
      int a = e % nj, c = e / nj;
      T acc = (T)0;
      for (int ri = 0; ri < r; ri++) acc += fb.E[a + (int64_t)ri * nj] * vR[ri * nrhs + c];
      if (shared && a >= k) {
        atomicAdd(v + fb.J[a] * nrhs + c, acc);  // near DOFs other boxes of the phase update too
        continue;
      }
      T nv = v[fb.J[a] * nrhs + c] + acc;
      v[fb.J[a] * nrhs + c] = nv;
      if (a < k) vS[a * nrhs + c] = nv;  // S is the head of J
    }
    __syncthreads();
    // U_T^{-1}: v_R += T^T v_S
    for (int e = tid; e < r * nrhs; e += NT) {
      int ri = e % r, c = e / r;
      T acc = (T)0;
      for (int q = 0; q < k; q++) acc += fb.Tm[q + (int64_t)ri * k] * vS[q * nrhs + c];
      v[Rr[ri] * nrhs + c] = vR[ri * nrhs + c] + acc;
    }
  }
}

// Solve sweeps (Eq. 3.11) for nrhs = NR <= 4 right-hand sides held in
// registers, with every box's rows split into chunks of SWEEP_CHUNK so that
// large boxes are spread over several CTAs.  The CTAs of one box meet at a
// per-box counter: the last to finish (no waiting) writes the box's own S
// and R entries, which every CTA of the box reads first, so the result does
// not depend on which CTA is last.
template <typename T, int NR>
__device__ __forceinline__ void sweep_gather(const FBox<T> &fb, const T *v, T *vS, T *vR) {
  const int k = fb.k, r = fb.r;
  for (int e = threadIdx.x; e < k * NR; e += NT) vS[e] = v[fb.ids[e / NR] * NR + e % NR];
  for (int e = threadIdx.x; e < r * NR; e += NT) vR[e] = v[fb.ids[k + e / NR] * NR + e % NR];
}

// Forward sweep (solve): tmp = v_R - T^T v_S; v_N -= E_N tmp over this CTA's
// chunk of J; the last CTA of the box: v_S -= E_S tmp, v_R = X_RR^{-1} tmp.
template <typename T, int NR>
__global__ void __launch_bounds__(NT) k_sweep_fwd(const FBox<T> *boxes, const int *wbox, const int *wchunk, T *v,
                                                  int *cnt, int shared) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  const int bi = wbox[blockIdx.x], ch = wchunk[blockIdx.x];
  const FBox<T> &fb = boxes[bi];
  const int k = fb.k, r = fb.r, nj = fb.nj;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T *vS = reinterpret_cast<T *>(smem_raw);  // k x NR
  T *vR = vS + (size_t)k * NR;               // r x NR
  T *tmp = vR + (size_t)r * NR;              // r x NR
  T *part = tmp + (size_t)r * NR;            // partial sums of X_RR^{-1} tmp
  sweep_gather<T, NR>(fb, v, vS, vR);
  __syncthreads();
  // tmp = v_R - T^T v_S: a warp per SWEEP_TROWS rows at once, so that the
  // loads of all of them are in flight together
  for (int ri0 = warp * SWEEP_TROWS; ri0 < r; ri0 += (NT / 32) * SWEEP_TROWS) {
    T acc[SWEEP_TROWS][NR];
#pragma unroll
    for (int u = 0; u < SWEEP_TROWS; u++)
#pragma unroll
      for (int c = 0; c < NR; c++) acc[u][c] = (T)0;
    for (int q = lane; q < k; q += 32) {
      T tq[SWEEP_TROWS];
#pragma unroll
      for (int u = 0; u < SWEEP_TROWS; u++) tq[u] = ri0 + u < r ? __ldg(fb.Tm + q + (int64_t)(ri0 + u) * k) : (T)0;
#pragma unroll
      for (int u = 0; u < SWEEP_TROWS; u++)
#pragma unroll
        for (int c = 0; c < NR; c++) acc[u][c] += tq[u] * vS[q * NR + c];
    }
#pragma unroll
    for (int u = 0; u < SWEEP_TROWS; u++)
#pragma unroll
      for (int c = 0; c < NR; c++) acc[u][c] = warp_sum(acc[u][c]);
    if (lane == 0)
#pragma unroll
      for (int u = 0; u < SWEEP_TROWS; u++)
        if (ri0 + u < r)
#pragma unroll
          for (int c = 0; c < NR; c++) tmp[(ri0 + u) * NR + c] = vR[(ri0 + u) * NR + c] - acc[u][c];
  }
  __syncthreads();
  // rows of E: two threads per row, each over alternate columns, SWEEP_MLP
  // loads in flight (the last group predicated); every lane of the warp
  // calls this (valid or not) for the final shuffle
  auto erow = [&](int a, bool valid, T *acc) {
    const T *ea = fb.E + a;
    const int h = tid & 1;
    for (int ri = valid ? h : r; ri < r; ri += 2 * SWEEP_MLP) {
      T ev[SWEEP_MLP];
#pragma unroll
      for (int u = 0; u < SWEEP_MLP; u++) ev[u] = ri + 2 * u < r ? __ldg(ea + (int64_t)(ri + 2 * u) * nj) : (T)0;
#pragma unroll
      for (int u = 0; u < SWEEP_MLP; u++)
        if (ri + 2 * u < r)
#pragma unroll
          for (int c = 0; c < NR; c++) acc[c] += ev[u] * tmp[(ri + 2 * u) * NR + c];
    }
#pragma unroll
    for (int c = 0; c < NR; c++) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 1);
  };
  {
    const int a = ch * SWEEP_CHUNK + (tid >> 1);
    T acc[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) acc[c] = (T)0;
    const bool mine = a < nj && a >= k;
    erow(a, a < nj, acc);
    if (mine && (tid & 1) == 0) {
      T *vg = v + fb.J[a] * NR;
      if (shared) {  // near DOFs other boxes of the phase update too
#pragma unroll
        for (int c = 0; c < NR; c++) atomicAdd(vg + c, -acc[c]);
      } else {
#pragma unroll
        for (int c = 0; c < NR; c++) vg[c] -= acc[c];
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    const int nchunk = max(1, (nj + SWEEP_CHUNK - 1) / SWEEP_CHUNK);
    s_last = atomicAdd(cnt + bi, 1) == nchunk - 1;
  }
  __syncthreads();
  if (!s_last) return;
  if (tid == 0) cnt[bi] = 0;
  // S rows of E (the head of J)
  for (int a0 = 0; a0 < k; a0 += NT / 2) {
    const int a = a0 + (tid >> 1);
    T acc[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) acc[c] = (T)0;
    erow(a, a < k, acc);
    if (a < k && (tid & 1) == 0) {
      T *vg = v + fb.ids[a] * NR;
#pragma unroll
      for (int c = 0; c < NR; c++) vg[c] = vS[a * NR + c] - acc[c];
    }
  }
  // D^{-1} on R: x_R = X_RR^{-1} tmp (rows split over nch groups of columns)
  const int nch = r >= NT ? 1 : NT / r;
  for (int i0 = 0; i0 < r; i0 += NT) {
    const int i = i0 + tid % (r >= NT ? NT : r), g = r >= NT ? 0 : tid / r;
    if (i < r && g < nch && tid < (r >= NT ? NT : nch * r)) {
      T acc[NR];
#pragma unroll
      for (int c = 0; c < NR; c++) acc[c] = (T)0;
      for (int l = g; l < r; l += SWEEP_MLP * nch) {
        T xv[SWEEP_MLP];
#pragma unroll
        for (int u = 0; u < SWEEP_MLP; u++) xv[u] = l + u * nch < r ? __ldg(fb.Xi + i + (int64_t)(l + u * nch) * r) : (T)0;
#pragma unroll
        for (int u = 0; u < SWEEP_MLP; u++)
          if (l + u * nch < r)
#pragma unroll
            for (int c = 0; c < NR; c++) acc[c] += xv[u] * tmp[(l + u * nch) * NR + c];
      }
#pragma unroll
      for (int c = 0; c < NR; c++) part[((size_t)g * r + i) * NR + c] = acc[c];
    }
  }
  __syncthreads();
  for (int i = tid; i < r; i += NT) {
    T *vg = v + fb.ids[k + i] * NR;
#pragma unroll
    for (int c = 0; c < NR; c++) {
      T sum = (T)0;
      for (int g = 0; g < nch; g++) sum += part[((size_t)g * r + i) * NR + c];
      vg[c] = sum;
    }
  }
}

// Backward sweep (solve): partial sums of G v_J over this CTA's chunk of J
// into pbuf; the last CTA of the box adds them in chunk order,
// v_R -= G v_J, v_S -= T v_R, and writes v_R and v_S.
template <typename T, int NR>
__global__ void __launch_bounds__(NT) k_sweep_bwd(const FBox<T> *boxes, const int *wbox, const int *wchunk, T *v,
                                                  int *cnt, T *pbuf, const int64_t *poff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  const int bi = wbox[blockIdx.x], ch = wchunk[blockIdx.x];
  const FBox<T> &fb = boxes[bi];
  const int k = fb.k, r = fb.r, nj = fb.nj;
  const int tid = threadIdx.x;
  T *part = reinterpret_cast<T *>(smem_raw);  // nch x r x NR, then vS, vR for the last CTA
  T *vJc = part + (size_t)NT * NR;             // this chunk's entries of v_J
  const int a0 = ch * SWEEP_CHUNK, a1 = min(nj, a0 + SWEEP_CHUNK), na = a1 - a0;
  const int nch = r >= NT ? 1 : NT / r;
  T *pb = pbuf + poff[bi] + (int64_t)ch * r * NR;
  // G(i, a) = gq[i * gsi + a * gsa]: the stored G, or E^T under symmetric storage
  const T *gq = fb.G ? fb.G : fb.E;
  const int64_t gsi = fb.G ? 1 : nj, gsa = fb.G ? r : 1;
  // the chunk's v_J gathered once, all loads in flight together
  for (int e = tid; e < na * NR; e += NT) vJc[e] = v[fb.J[a0 + e / NR] * NR + e % NR];
  __syncthreads();
  for (int i0 = 0; i0 < r; i0 += NT) {
    const int rr = r >= NT ? NT : r;
    const int i = i0 + tid % rr, g = tid / rr;
    if (i < r && g < nch) {
      T acc[NR];
#pragma unroll
      for (int c = 0; c < NR; c++) acc[c] = (T)0;
      const T *gi = gq + i * gsi + a0 * gsa;
      for (int a = g; a < na; a += SWEEP_MLP * nch) {
        T gv[SWEEP_MLP];
#pragma unroll
        for (int u = 0; u < SWEEP_MLP; u++) gv[u] = a + u * nch < na ? __ldg(gi + (a + u * nch) * gsa) : (T)0;
#pragma unroll
        for (int u = 0; u < SWEEP_MLP; u++)
          if (a + u * nch < na)
#pragma unroll
            for (int c = 0; c < NR; c++) acc[c] += gv[u] * vJc[(a + u * nch) * NR + c];
      }
#pragma unroll
      for (int c = 0; c < NR; c++) part[((size_t)g * rr + (i - i0)) * NR + c] = acc[c];
    }
    __syncthreads();
    for (int e = tid; e < (r - i0 < rr ? r - i0 : rr) * NR; e += NT) {
      const int il = e / NR, c = e % NR;
      T sum = (T)0;
      for (int g2 = 0; g2 < nch; g2++) sum += part[((size_t)g2 * rr + il) * NR + c];
      pb[(int64_t)(i0 + il) * NR + c] = sum;
    }
    __syncthreads();
  }
  __threadfence();
  if (tid == 0) {
    const int nchunk = max(1, (nj + SWEEP_CHUNK - 1) / SWEEP_CHUNK);
    s_last = atomicAdd(cnt + bi, 1) == nchunk - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid == 0) cnt[bi] = 0;
  const int nchunk = max(1, (nj + SWEEP_CHUNK - 1) / SWEEP_CHUNK);
  T *vS = part, *vR = part + (size_t)k * NR;
  sweep_gather<T, NR>(fb, v, vS, vR);
  __syncthreads();
  const T *p0 = pbuf + poff[bi];
  for (int e = tid; e < r * NR; e += NT) {
    T sum = (T)0;
    for (int c2 = 0; c2 < nchunk; c2++) sum += __ldcg(p0 + (int64_t)c2 * r * NR + e);
    vR[e] -= sum;
  }
  __syncthreads();
  // v_S -= T v_R: the columns of T split over nq groups of threads
  // (SWEEP_MLP loads in flight each), the groups' partial sums added in group order
  if (k > 0) {
    const int kk = k >= NT ? NT : k, nq = k >= NT ? 1 : NT / k;
    T *tp = part + (size_t)(k + r) * NR;  // nq x kk x NR partial sums
    for (int q0 = 0; q0 < k; q0 += NT) {
      const int q = q0 + tid % kk, g = tid / kk;
      if (q < k && g < nq) {
        T acc[NR];
#pragma unroll
        for (int c = 0; c < NR; c++) acc[c] = (T)0;
        for (int ri = g; ri < r; ri += SWEEP_MLP * nq) {
          T tv[SWEEP_MLP];
#pragma unroll
          for (int u = 0; u < SWEEP_MLP; u++) tv[u] = ri + u * nq < r ? __ldg(fb.Tm + q + (int64_t)(ri + u * nq) * k) : (T)0;
#pragma unroll
          for (int u = 0; u < SWEEP_MLP; u++)
            if (ri + u * nq < r)
#pragma unroll
              for (int c = 0; c < NR; c++) acc[c] += tv[u] * vR[(ri + u * nq) * NR + c];
        }
#pragma unroll
        for (int c = 0; c < NR; c++) tp[((size_t)g * kk + (q - q0)) * NR + c] = acc[c];
      }
      __syncthreads();
      for (int e = tid; e < min(kk, k - q0) * NR; e += NT) {
        const int ql = e / NR, c = e % NR;
        T sum = (T)0;
        for (int g2 = 0; g2 < nq; g2++) sum += tp[((size_t)g2 * kk + ql) * NR + c];
        v[fb.ids[q0 + ql] * NR + c] = vS[(q0 + ql) * NR + c] - sum;
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < r * NR; e += NT) v[fb.ids[k + e / NR] * NR + e % NR] = vR[e];
}

template <typename T>
void launch_sweep_chunks(int mode, const FBox<T> *boxes, const int *wbox, const int *wchunk, int nwork, T *v,
                         int nrhs, int bmax, int *cnt, T *pbuf, const int64_t *poff, cudaStream_t st, int shared) {
  if (nwork == 0) return;
  const size_t smem = sweep_chunk_smem(bmax, nrhs, (int)sizeof(T));
  constexpr int SMAX = (200 << 10) + 64;  // callers keep smem within this
#define RSS_SWEEP_NR(NRV)                                                                                   \
  case NRV:                                                                                                \
    if (mode == SWEEP_SOLVE_FWD) {                                                                         \
      if (!capturing(st)) cudaFuncSetAttribute(k_sweep_fwd<T, NRV>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMAX); \
      k_sweep_fwd<T, NRV><<<nwork, NT, smem, st>>>(boxes, wbox, wchunk, v, cnt, shared);                           \
    } else {                                                                                               \
      if (!capturing(st)) cudaFuncSetAttribute(k_sweep_bwd<T, NRV>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMAX); \
      k_sweep_bwd<T, NRV><<<nwork, NT, smem, st>>>(boxes, wbox, wchunk, v, cnt, pbuf, poff);               \
    }                                                                                                      \
    break;
  switch (nrhs) {
    RSS_SWEEP_NR(1)
    RSS_SWEEP_NR(2)
    RSS_SWEEP_NR(3)
    RSS_SWEEP_NR(4)
  }
#undef RSS_SWEEP_NR
  count_launch();
}

size_t sweep_chunk_smem(int bmax, int nrhs, int elem) {
  return ((size_t)4 * bmax + NT + SWEEP_CHUNK) * nrhs * elem + 64;
}

template <typename T>
void launch_sweep(int mode, const FBox<T> *boxes, int first, int count, T *v, int nrhs, int bmax, int njmax,
                  cudaStream_t st, int shared) {
  if (count == 0) return;
  const bool force_general = njmax < 0;  // large-box path requested
  if (force_general) njmax = -njmax;
  size_t smem = ((size_t)3 * bmax + (size_t)njmax) * nrhs * sizeof(T) + 64;
  int jsh = 1;
  if (smem > (size_t)(200 << 10) || force_general) {
    jsh = 0;
    smem = (size_t)3 * bmax * nrhs * sizeof(T) + 64;
  }
  if (!capturing(st)) cudaFuncSetAttribute(k_sweep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (200 << 10) + 64);
  k_sweep<T><<<count, NT, smem, st>>>(mode, boxes, first, v, nrhs, jsh, shared); count_launch();
}

// ---------------------------------------------------------------------------
// Generalized square root F^{1/2} (the remark after Eq. 3.11): Cholesky
// factors of the diagonal blocks of D, rebuilt from their stored LU factors
// ---------------------------------------------------------------------------

// Block q of `nblk` (the boxes' X_RR, then the problems' top blocks): its LU
// (row-major, P X = L U, row i of P X is row piv[i] of X), order r, and the
// place of its Cholesky factor.  One CTA per block: X = P^T L U is formed in
// C, then C := the lower Cholesky factor of (X + X^T) / 2 in place, column
// by column (the upper triangle still holds X until it is cleared).  A block
// that is not positive definite records DERR_NUMERIC.
template <typename T>
__global__ void __launch_bounds__(NT) k_chol_from_lu(const FBox<T> *boxes, int nbox, const T *topLU,
                                                     const int64_t *loff, const int *toppiv, const int64_t *toff,
                                                     const int *tn, T *Call, const int64_t *coff, int *err) {
  const int q = blockIdx.x, tid = threadIdx.x;
  const T *LU;
  const int *piv;
  int r;
  if (q < nbox) {
    LU = boxes[q].LU;
    piv = boxes[q].piv;
    r = boxes[q].r;
  } else {
    const int p = q - nbox;
    LU = topLU + loff[p];
    piv = toppiv + toff[p];
    r = tn[p];
  }
  if (r == 0) return;
  T *C = Call + coff[q];
  for (int e = tid; e < r * r; e += NT) {
    const int i = e / r, j = e % r, m = i < j ? i : j;
    T acc = (T)0;
    for (int l = 0; l <= m; l++) acc += (l == i ? (T)1 : LU[(int64_t)i * r + l]) * LU[(int64_t)l * r + j];
    C[(int64_t)piv[i] * r + j] = acc;
  }
  __syncthreads();
  __shared__ T s_d;
  for (int j = 0; j < r; j++) {
    if (tid == 0) {
      T d = C[(int64_t)j * r + j];
      for (int l = 0; l < j; l++) d -= C[(int64_t)j * r + l] * C[(int64_t)j * r + l];
      if (!(d > (T)0)) {
        set_err(err, DERR_NUMERIC);
        d = (T)1;  // keep going with a harmless pivot; the host reports the error
      }
      s_d = sqrt(d);
      C[(int64_t)j * r + j] = s_d;
    }
    __syncthreads();
    const T dj = s_d;
    for (int i = j + 1 + tid; i < r; i += NT) {
      T acc = (T)0.5 * (C[(int64_t)i * r + j] + C[(int64_t)j * r + i]);
      for (int l = 0; l < j; l++) acc -= C[(int64_t)i * r + l] * C[(int64_t)j * r + l];
      C[(int64_t)i * r + j] = acc / dj;
    }
    __syncthreads();
  }
  for (int e = tid; e < r * r; e += NT) {
    const int i = e / r, j = e % r;
    if (i < j) C[e] = (T)0;
  }
}

// v_B := C v_B (trans = 0) or C^T v_B (trans = 1) on every block's DOFs (a
// box's R, a problem's top-block DOFs), C its lower Cholesky factor.
template <typename T>
__global__ void __launch_bounds__(NT) k_chol_apply(const FBox<T> *boxes, int nbox, const int64_t *top,
                                                   const int64_t *toff, const int *tn, const T *Call,
                                                   const int64_t *coff, T *v, int nrhs, int trans) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const int q = blockIdx.x, tid = threadIdx.x;
  const int64_t *ids;
  int r;
  if (q < nbox) {
    ids = boxes[q].ids + boxes[q].k;
    r = boxes[q].r;
  } else {
    const int p = q - nbox;
    ids = top + toff[p];
    r = tn[p];
  }
  if (r == 0) return;
  const T *C = Call + coff[q];
  for (int e = tid; e < r * nrhs; e += NT) xs[e] = v[ids[e / nrhs] * nrhs + e % nrhs];
  __syncthreads();
  for (int e = tid; e < r * nrhs; e += NT) {
    const int a = e / nrhs, c = e % nrhs;
    T acc = (T)0;
    if (!trans)
      for (int l = 0; l <= a; l++) acc += C[(int64_t)a * r + l] * xs[l * nrhs + c];
    else
      for (int l = a; l < r; l++) acc += C[(int64_t)l * r + a] * xs[l * nrhs + c];
    v[ids[a] * nrhs + c] = acc;
  }
}

template <typename T>
void launch_chol_from_lu(const FBox<T> *boxes, int nbox, const T *topLU, const int64_t *loff, const int *toppiv,
                         const int64_t *toff, const int *tn, int nprob, T *C, const int64_t *coff, int *err,
                         cudaStream_t st) {
  if (nbox + nprob == 0) return;
  k_chol_from_lu<T><<<nbox + nprob, NT, 0, st>>>(boxes, nbox, topLU, loff, toppiv, toff, tn, C, coff, err);
  count_launch();
}

template <typename T>
void launch_chol_apply(const FBox<T> *boxes, int nbox, const int64_t *top, const int64_t *toff, const int *tn,
                       int nprob, const T *C, const int64_t *coff, T *v, int nrhs, int rmax, int trans,
                       cudaStream_t st) {
  if (nbox + nprob == 0) return;
  const size_t smem = (size_t)rmax * nrhs * sizeof(T) + 16;
  if (!capturing(st)) cudaFuncSetAttribute(k_chol_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_chol_apply<T><<<nbox + nprob, NT, smem, st>>>(boxes, nbox, top, toff, tn, C, coff, v, nrhs, trans);
  count_launch();
}

// Raise the dynamic shared-memory limit of every sweep kernel on the current
// device (both element types, every right-hand-side count of the chunked
// forms), so that later launches need no attribute call, for instance while a
// stream is being captured.
void sweep_kernel_attributes() {
  constexpr int SMAX = (200 << 10) + 64;
  cudaFuncSetAttribute(k_sweep<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMAX);
  cudaFuncSetAttribute(k_sweep<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMAX);
#define RSS_SWEEP_ATTR(TT, NRV)                                                                   \
  cudaFuncSetAttribute(k_sweep_fwd<TT, NRV>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMAX); \
  cudaFuncSetAttribute(k_sweep_bwd<TT, NRV>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMAX);
  RSS_SWEEP_ATTR(float, 1) RSS_SWEEP_ATTR(float, 2) RSS_SWEEP_ATTR(float, 3) RSS_SWEEP_ATTR(float, 4)
  RSS_SWEEP_ATTR(double, 1) RSS_SWEEP_ATTR(double, 2) RSS_SWEEP_ATTR(double, 3) RSS_SWEEP_ATTR(double, 4)
#undef RSS_SWEEP_ATTR
}

// Top blocks of one or more problems (Sec. 3.3.3): problem p has tn[p] DOFs
// with global ids top[toff[p] ...], its LU (row-major, P A = L U) at
// LU + loff[p] and pivots at piv + toff[p].  Solve (mode 0) or multiply
// (mode 1); one CTA per (problem, right-hand side).
template <typename T>
__global__ void __launch_bounds__(1024) k_top(int mode, const T *LUall, const int64_t *loff, const int *pivall,
                                              const int64_t *topall, const int64_t *toff, const int *tn, T *v,
                                              int nrhs, T *work) {
  const int p = blockIdx.x / nrhs, c = blockIdx.x % nrhs;
  const int n = tn[p];
  if (n == 0) return;
  const T *LU = LUall + loff[p];
  const int *piv = pivall + toff[p];
  const int64_t *top = topall + toff[p];
  T *y = work + 2 * (toff[p] * nrhs + (int64_t)c * n);
  T *u = y + n;
  const int tid = threadIdx.x;
  if (mode == 0) {
    for (int i = tid; i < n; i += blockDim.x) y[i] = v[top[piv[i]] * nrhs + c];
    __syncthreads();
    for (int i = 0; i < n; i++) {
      T yi = y[i];
      for (int l = i + 1 + tid; l < n; l += blockDim.x) y[l] -= LU[(int64_t)l * n + i] * yi;
      __syncthreads();
    }
    for (int i = n - 1; i >= 0; i--) {
      T yi = y[i] / LU[(int64_t)i * n + i];
      __syncthreads();
      if (tid == 0) y[i] = yi;
      for (int l = tid; l < i; l += blockDim.x) y[l] -= LU[(int64_t)l * n + i] * yi;
      __syncthreads();
    }
    for (int i = tid; i < n; i += blockDim.x) v[top[i] * nrhs + c] = y[i];
  } else {
    for (int i = tid; i < n; i += blockDim.x) y[i] = v[top[i] * nrhs + c];
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
      T s = (T)0;
      for (int l = i; l < n; l++) s += LU[(int64_t)i * n + l] * y[l];
      u[i] = s;
    }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
      T s = u[i];
      for (int l = 0; l < i; l++) s += LU[(int64_t)i * n + l] * u[l];
      v[top[piv[i]] * nrhs + c] = s;
    }
  }
}

// W = U^{-1} L^{-1} for one top block's LU (row-major; unit lower L below
// the diagonal, U on and above), so that the solve's D^{-1} on the top
// block is W (P v), a matrix-vector product, instead of two triangular
// sweeps with a barrier per row.  One warp per column k of W: z = L^{-1}
// e_k, then U^{-1} z, each row's dot product spread over the lanes; z in
// shared memory.  Columns are independent, so the warps never wait on one
// another.
constexpr int TOPINV_WARPS = 4;
template <typename T> __global__ void __launch_bounds__(32 * TOPINV_WARPS) k_top_inverse(const T *LU, int n, T *W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = blockIdx.x * TOPINV_WARPS + w;
  if (k >= n) return;  // the whole warp: no barrier follows
  T *z = reinterpret_cast<T *>(smem_raw) + (size_t)w * n;
  for (int i = lane; i < n; i += 32) z[i] = i == k ? (T)1 : (T)0;
  __syncwarp();
  for (int i = k + 1; i < n; i++) {
    const T *Li = LU + (int64_t)i * n;
    T acc = (T)0;
    for (int l = k + lane; l < i; l += 32) acc += Li[l] * z[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[i] = -acc;
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; i--) {
    const T *Ui = LU + (int64_t)i * n;
    T acc = (T)0;
    for (int l = i + 1 + lane; l < n; l += 32) acc += Ui[l] * z[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[i] = (z[i] - acc) / Ui[i];
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) W[(int64_t)i * n + k] = z[i];
}

template <typename T> void launch_top_inverse(const T *LU, int n, T *W, cudaStream_t st) {
  if (n == 0) return;
  k_top_inverse<T><<<(n + TOPINV_WARPS - 1) / TOPINV_WARPS, 32 * TOPINV_WARPS,
                     (size_t)TOPINV_WARPS * n * sizeof(T), st>>>(LU, n, W);
  count_launch();
}

// y = P v_top (the pivoted gather), then v_top = W y with one warp per row.
template <typename T>
__global__ void k_top_gather(const int *piv, const int64_t *top, int n, const T *v, int nrhs, T *y) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  const int kk = e / nrhs, c = e - kk * nrhs;
  y[e] = v[top[piv[kk]] * nrhs + c];
}
template <typename T, int NR>
__global__ void __launch_bounds__(256) k_top_gemv(const T *W, const int64_t *top, int n, const T *y, T *v) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n) return;
  const T *Wi = W + (int64_t)i * n;
  T acc[NR];
#pragma unroll
  for (int c = 0; c < NR; c++) acc[c] = (T)0;
  for (int kk = lane; kk < n; kk += 32) {
    const T w = Wi[kk];
#pragma unroll
    for (int c = 0; c < NR; c++) acc[c] += w * y[kk * NR + c];
  }
#pragma unroll
  for (int c = 0; c < NR; c++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < NR; c++) v[top[i] * NR + c] = acc[c];
}

template <typename T>
void launch_top(int mode, const T *LU, const int64_t *loff, const int *piv, const int64_t *top, const int64_t *toff,
                const int *tn, int nprob, int ntop_total, T *v, int nrhs, T *work, cudaStream_t st, const T *Winv) {
  if (ntop_total == 0 || nprob == 0) return;
  if (mode == 0 && Winv && nprob == 1 && nrhs >= 1 && nrhs <= 4) {
    const int n = ntop_total;
    k_top_gather<T><<<(n * nrhs + 255) / 256, 256, 0, st>>>(piv, top, n, v, nrhs, work);
    count_launch();
    const unsigned g = (unsigned)((n + 7) / 8);
    if (nrhs == 1) k_top_gemv<T, 1><<<g, 256, 0, st>>>(Winv, top, n, work, v);
    else if (nrhs == 2) k_top_gemv<T, 2><<<g, 256, 0, st>>>(Winv, top, n, work, v);
    else if (nrhs == 3) k_top_gemv<T, 3><<<g, 256, 0, st>>>(Winv, top, n, work, v);
    else k_top_gemv<T, 4><<<g, 256, 0, st>>>(Winv, top, n, work, v);
    count_launch();
    return;
  }
  k_top<T><<<nprob * nrhs, 1024, 0, st>>>(mode, LU, loff, piv, top, toff, tn, v, nrhs, work);
  count_launch();
}

// LU with partial pivoting of many small dense blocks, one CTA per block
// (row-major, in place; pivot = largest |entry|, ties to the lowest row).
template <typename T>
__global__ void __launch_bounds__(256) k_lu_batched(T *LUall, const int64_t *loff, int *pivall, const int64_t *toff,
                                                    const int *tn, int *err) {
  __shared__ T s_val[8];
  __shared__ int s_idx[8];
  const int p = blockIdx.x, n = tn[p];
  T *A = LUall + loff[p];
  int *piv = pivall + toff[p];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += blockDim.x) piv[i] = i;
  __syncthreads();
  for (int j = 0; j < n; j++) {
    T best = (T)-1;
    int bi = n;
    for (int i = j + tid; i < n; i += blockDim.x) {
      T v = fabs(A[(int64_t)i * n + j]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      s_val[warp] = best;
      s_idx[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      for (int u = 1; u < (int)(blockDim.x >> 5); u++)
        if (s_val[u] > best || (s_val[u] == best && s_idx[u] < bi)) {
          best = s_val[u];
          bi = s_idx[u];
        }
      if (bi >= n) {
        bi = j;
        set_err(err, DERR_NUMERIC);
      }
      if (best == (T)0) set_err(err, DERR_NUMERIC);
      s_idx[0] = bi;
    }
    __syncthreads();
    const int pr = s_idx[0];
    if (pr != j) {
      for (int cc = tid; cc < n; cc += blockDim.x) {
        T t0 = A[(int64_t)j * n + cc];
        A[(int64_t)j * n + cc] = A[(int64_t)pr * n + cc];
        A[(int64_t)pr * n + cc] = t0;
      }
      if (tid == 0) {
        int tp = piv[j];
        piv[j] = piv[pr];
        piv[pr] = tp;
      }
    }
    __syncthreads();
    const T d = A[(int64_t)j * n + j];
    for (int i = j + 1 + tid; i < n; i += blockDim.x) A[(int64_t)i * n + j] /= d;
    __syncthreads();
    const int rem = n - j - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      int i = j + 1 + e / rem, cc = j + 1 + e % rem;
      A[(int64_t)i * n + cc] -= A[(int64_t)i * n + j] * A[(int64_t)j * n + cc];
    }
    __syncthreads();
  }
}

template <typename T>
void launch_lu_batched(T *LU, const int64_t *loff, int *piv, const int64_t *toff, const int *tn, int nprob,
                       cudaStream_t st, int *err) {
  if (nprob == 0) return;
  k_lu_batched<T><<<nprob, 256, 0, st>>>(LU, loff, piv, toff, tn, err);
  count_launch();
}

// dir 0: out_t[g*nrhs+c] = in[perm[g] + c*n];  dir 1: out[perm[g] + c*n] = in_t[g*nrhs+c]
template <typename T>
__global__ void k_permute(int dir, const int64_t *perm, const double *in, T *tv, double *out, int64_t n,
                          int nrhs) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  int64_t g = e / nrhs;
  int c = (int)(e % nrhs);
  if (dir == 0)
    tv[e] = (T)in[perm[g] + (int64_t)c * n];
  else
    out[perm[g] + (int64_t)c * n] = (double)tv[e];
}

template <typename T>
void launch_permute(int dir, const int64_t *perm, const double *in, T *tv, double *out, int64_t n, int nrhs,
                    cudaStream_t st) {
  int64_t tot = n * nrhs;
  if (tot == 0) return;
  k_permute<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(dir, perm, in, tv, out, n, nrhs); count_launch();
}

// Natural logarithm by Tang's table-driven method (P. T. P. Tang, ACM Trans.
// Math. Softw. 16(4), 1990): x = 2^e m with m in [1, 2) read from the bits;
// c = 1 + (2k + 1) / 256 is the centre of m's interval of width 1/128 (k
// the top 7 bits of m's fraction), so log x = e ln 2 + log c + log(1 + t)
// with t = (m - c) / c, |t| < 2^-8 (m - c is exact); log(1 + t) is its
// Taylor series to t^6 (the first term left out is below 2^-58).
// tab[k] = (1 / c, log c).  The absolute error is a few units of 2^-53
// times max(1, |log x|).  Zero, negative, subnormal and non-finite x take
// log() itself.
__device__ __forceinline__ double log_tab(double x, const double2 *tab) {
  const long long u = __double_as_longlong(x);
  const int ef = (int)((u >> 52) & 0x7ff);
  if (!(x > 0.0) || ef == 0 || ef == 0x7ff) return log(x);
  const int k = (int)((u >> 45) & 127);
  const double m = __longlong_as_double((u & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  const double c = 1.0 + (double)(2 * k + 1) * (1.0 / 256.0);
  const double2 fl = tab[k];
  const double t = (m - c) * fl.x;
  // log(1 + t) = t + t^2 (-1/2 + t/3 - t^2/4 + t^3/5 - t^4/6)
  double qv = fma(t, -1.0 / 6.0, 1.0 / 5.0);
  qv = fma(t, qv, -0.25);
  qv = fma(t, qv, 1.0 / 3.0);
  qv = fma(t, qv, -0.5);
  const double l1p = fma(t * t, qv, t);
  return fma((double)(ef - 1023), 0.69314718055994530942, fl.y + l1p);
}

// Exact FP64 y = A x by direct summation (tree-ordered points, caller-order
// vectors through perm), for one or several independent problems: tile q
// covers targets [tstart[q], tend[q]) of a problem whose DOFs are
// [sbeg[q], send[q]); sources are staged in shared memory.  Each point's
// weight comes from wdof (or K.w).  The 2D kernel's logarithm is log_tab's.
__global__ void __launch_bounds__(256) k_matvec(const double *xt, int dim, KernelParams K, const double *wdof,
                                                const int64_t *perm, const double *xin, double *yout, int64_t n,
                                                int nrhs, const int64_t *tstart, const int64_t *tend,
                                                const int64_t *sbeg, const int64_t *send) {
  __shared__ double sp[256 * 3];
  __shared__ double sx[256 * 4];
  __shared__ double2 s_logtab[128];
  if (threadIdx.x < 128) {
    const double c = 1.0 + (double)(2 * threadIdx.x + 1) * (1.0 / 256.0);
    s_logtab[threadIdx.x] = make_double2(1.0 / c, log(c));
  }
  __syncthreads();
  const int q = blockIdx.x;
  const int64_t i = tstart[q] + threadIdx.x;
  const bool live = i < tend[q];
  const int64_t j0b = sbeg[q], j1b = send[q];
  const int cb = blockIdx.y * 4;
  const int nc = min(4, nrhs - cb);
  double xi[3] = {0, 0, 0};
  double w = K.w;
  if (live) {
    for (int d = 0; d < dim; d++) xi[d] = xt[i * dim + d];
    if (wdof) w = wdof[i];
  }
  double acc[4] = {0, 0, 0, 0};
  for (int64_t j0 = j0b; j0 < j1b; j0 += 256) {
    int64_t j = j0 + threadIdx.x;
    if (j < j1b) {
      for (int d = 0; d < dim; d++) sp[threadIdx.x * 3 + d] = xt[j * dim + d];
      for (int c = 0; c < nc; c++) sx[threadIdx.x * 4 + c] = xin[perm[j] + (int64_t)(cb + c) * n];
    }
    __syncthreads();
    int lim = (int)min((int64_t)256, j1b - j0);
    if (live) {
      for (int qq = 0; qq < lim; qq++) {
        int64_t jj = j0 + qq;
        double a;
        if (jj == i) {
          a = K.diag;
        } else {
          double r2 = 0.0;
          for (int d = 0; d < dim; d++) {
            double z = xi[d] - sp[qq * 3 + d];
            r2 += z * z;
          }
          a = w * (K.kind == 0 ? -log_tab(r2, s_logtab) * (1.0 / (4.0 * kPi)) : (1.0 / (4.0 * kPi)) / sqrt(r2));
        }
        for (int c = 0; c < nc; c++) acc[c] += a * sx[qq * 4 + c];
      }
    }
    __syncthreads();
  }
  if (live)
    for (int c = 0; c < nc; c++) yout[perm[i] + (int64_t)(cb + c) * n] = acc[c];
}

void launch_matvec(const double *x_tree, int dim, const KernelParams &K, const double *wdof, const int64_t *perm,
                   const double *xin, double *yout, int64_t n, int nrhs, int ntile, const int64_t *tstart,
                   const int64_t *tend, const int64_t *sbeg, const int64_t *send, cudaStream_t st) {
  if (n == 0 || ntile == 0) return;
  dim3 g((unsigned)ntile, (nrhs + 3) / 4);
  k_matvec<<<g, 256, 0, st>>>(x_tree, dim, K, wdof, perm, xin, yout, n, nrhs, tstart, tend, sbeg, send);
  count_launch();
}

// y = A x with the kernel evaluated in FP32 (tiles as k_matvec; the
// sources' depth-20 cells and offsets staged in shared memory; each tile's
// 256 terms summed in FP32, the tiles' sums in FP64).
__global__ void __launch_bounds__(256) k_matvec_f32(Points P, int kind, float wk, float diag, const int64_t *perm,
                                                    const double *xin, double *yout, int64_t n, int nrhs,
                                                    const int64_t *tstart, const int64_t *tend,
                                                    const int64_t *sbeg, const int64_t *send) {
  __shared__ int sc[256 * 3];
  __shared__ float so[256 * 3];
  __shared__ float sx[256 * 4];
  const int q = blockIdx.x, dim = P.dim;
  const int64_t i = tstart[q] + threadIdx.x;
  const bool live = i < tend[q];
  const int64_t j0b = sbeg[q], j1b = send[q];
  const int cb = blockIdx.y * 4;
  const int nc = min(4, nrhs - cb);
  int ci[3] = {0, 0, 0};
  float oi[3] = {0.f, 0.f, 0.f};
  float w = wk;
  if (live) {
    for (int d = 0; d < dim; d++) ci[d] = P.cell[3 * i + d], oi[d] = P.off[3 * i + d];
    if (P.wdof) w = (float)P.wdof[i];
  }
  double acc[4] = {0, 0, 0, 0};
  for (int64_t j0 = j0b; j0 < j1b; j0 += 256) {
    const int64_t j = j0 + threadIdx.x;
    if (j < j1b) {
      for (int d = 0; d < dim; d++) sc[threadIdx.x * 3 + d] = P.cell[3 * j + d], so[threadIdx.x * 3 + d] = P.off[3 * j + d];
      for (int c = 0; c < nc; c++) sx[threadIdx.x * 4 + c] = (float)xin[perm[j] + (int64_t)(cb + c) * n];
    }
    __syncthreads();
    const int lim = (int)min((int64_t)256, j1b - j0);
    if (live) {
      float t[4] = {0.f, 0.f, 0.f, 0.f};
      const int self = (i >= j0 && i < j0 + lim) ? (int)(i - j0) : -1;
      for (int qq = 0; qq < lim; qq++) {
        float r2 = 0.f;
        for (int d = 0; d < dim; d++) {
          const float z = fmaf((float)(ci[d] - sc[qq * 3 + d]), P.D, oi[d] - so[qq * 3 + d]);
          r2 = fmaf(z, z, r2);
        }
        const float a = qq == self ? diag : w * kof(kind, r2);
        for (int c = 0; c < nc; c++) t[c] = fmaf(a, sx[qq * 4 + c], t[c]);
      }
      for (int c = 0; c < nc; c++) acc[c] += (double)t[c];
    }
    __syncthreads();
  }
  if (live)
    for (int c = 0; c < nc; c++) yout[perm[i] + (int64_t)(cb + c) * n] = acc[c];
}

void launch_matvec_f32(const Points &P, const KernelParams &K, const int64_t *perm, const double *xin,
                       double *yout, int64_t n, int nrhs, int ntile, const int64_t *tstart, const int64_t *tend,
                       const int64_t *sbeg, const int64_t *send, cudaStream_t st) {
  if (n == 0 || ntile == 0) return;
  dim3 g((unsigned)ntile, (nrhs + 3) / 4);
  k_matvec_f32<<<g, 256, 0, st>>>(P, K.kind, (float)K.w, (float)K.diag, perm, xin, yout, n, nrhs, tstart, tend,
                                  sbeg, send);
  count_launch();
}

// ---------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------
#define RSS_INST(T)                                                                                          \
  template void launch_assemble<T>(const AssembleList &, T *, const LevelDev<T> *, const Points &,             \
                                   const KernelParams &, int64_t, cudaStream_t);                              \
  template void launch_id<T>(const LevelDev<T> &, FBox<T> *, const int *, int, int, int, const Points &,       \
                             const KernelParams &, const ProxyParams &, const T *, double, T *, int64_t, bool,       \
                             cudaStream_t,                                                                   \
                             int *);                                                                          \
  template void launch_elim<T>(const LevelDev<T> &, FBox<T> *, const int *, int, int, T *, int64_t,            \
                               const Overflow<T> &, cudaStream_t, int *, int);                                \
  template void launch_schur<T>(const LevelDev<T> &, const FBox<T> *, const int *, int, int, const T *, int64_t, \
                                cudaStream_t);                                                                \
  template void launch_dense_lu<T>(T *, int, int *, T *, cudaStream_t, int *);                                     \
  template void launch_sweep<T>(int, const FBox<T> *, int, int, T *, int, int, int, cudaStream_t, int);       \
  template void launch_sweep_chunks<T>(int, const FBox<T> *, const int *, const int *, int, T *, int, int, int *, \
                                       T *, const int64_t *, cudaStream_t, int);                             \
  template void launch_chol_from_lu<T>(const FBox<T> *, int, const T *, const int64_t *, const int *,            \
                                       const int64_t *, const int *, int, T *, const int64_t *, int *, cudaStream_t); \
  template void launch_chol_apply<T>(const FBox<T> *, int, const int64_t *, const int64_t *, const int *, int,     \
                                     const T *, const int64_t *, T *, int, int, int, cudaStream_t);              \
  template void launch_top<T>(int, const T *, const int64_t *, const int *, const int64_t *, const int64_t *,     \
                             const int *, int, int, T *, int, T *, cudaStream_t, const T *);                 \
  template void launch_top_inverse<T>(const T *, int, T *, cudaStream_t);                                     \
  template void launch_lu_batched<T>(T *, const int64_t *, int *, const int64_t *, const int *, int, cudaStream_t, \
                                     int *);                                                                  \
  template void launch_permute<T>(int, const int64_t *, const double *, T *, double *, int64_t, int,          \
                                  cudaStream_t);
RSS_INST(float)
RSS_INST(double)

}  // namespace rss
