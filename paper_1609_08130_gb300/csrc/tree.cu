// tree.cu -- the adaptive 2^d-tree of the factorization (Sec. 3: boxes are
// split until every leaf holds at most leaf_size points; Sec. 4: refined to
// n_occ points per leaf) built on the GPU.
//
// The tree is the one a recursive split produces: root [0,1]^d, a node of
// depth t splits iff it holds more than leaf_size points and t < 20; the
// integer cell of coordinate v at depth t is floor(v 2^t) clamped to
// [0, 2^t - 1]; child index sum_d bit_d << d; DOFs in stable pre-order
// (children ascending, points of a leaf in original order); nodes numbered
// in pre-order.  It is computed without recursion:
//   1. every point's depth-20 cell and Morton key (x in the lowest bit of each
//      group of d bits, a problem index above the 20 d key bits when several
//      problems share the build);
//   2. a stable LSD radix sort of (key, index) -- a depth-t node is a run of
//      points sharing the key's top d t bits, and the runs come out in child
//      order;
//   3. a point's leaf depth L is the first depth at which its run holds at
//      most leaf_size points (or 20): found by bisection on the depth, each
//      run's extent by binary search in the sorted keys;
//   4. a node of depth t starts at point p iff p starts a depth-t run and
//      t <= L(p); the depths at which p starts a run are t_b(p) .. 20, t_b
//      given by the highest bit where p's key differs from its predecessor's,
//      so p starts nodes at depths t_b(p) .. L(p), and pre-order numbering is
//      the order of (start, depth): an exclusive scan of the per-point node
//      counts;
//   5. within a leaf shallower than 20, the points are put back in original
//      order (a rank sort of at most leaf_size indices).
#include <cuda_runtime.h>

#include <utility>

#include "internal.h"

namespace rss {

namespace {

constexpr int RS_T = 256;              // threads per radix-sort block
constexpr int RS_ITEMS = 8;            // sub-tiles of RS_T keys per block
constexpr int RS_TILE = RS_T * RS_ITEMS;
constexpr int MAXD = 20;               // maximum depth of the tree

__device__ __forceinline__ uint64_t spread2(uint64_t x) {
  x &= 0x1fffffULL;
  x = (x | (x << 16)) & 0x0000ffff0000ffffULL;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffULL;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0fULL;
  x = (x | (x << 2)) & 0x3333333333333333ULL;
  x = (x | (x << 1)) & 0x5555555555555555ULL;
  return x;
}
__device__ __forceinline__ uint64_t spread3(uint64_t x) {
  x &= 0x1fffffULL;
  x = (x | (x << 32)) & 0x001f00000000ffffULL;
  x = (x | (x << 16)) & 0x001f0000ff0000ffULL;
  x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
  x = (x | (x << 2)) & 0x1249249249249249ULL;
  return x;
}

// Depth-20 cells, Morton keys and point indices.  pofs (nprob + 1 entries)
// gives each problem's first point; the problem index goes above the key.
__global__ void k_tree_keys(const double *__restrict__ pts, int64_t n, int dim, const int64_t *__restrict__ pofs,
                            int nprob, uint64_t *__restrict__ key, uint64_t *__restrict__ mkey,
                            int64_t *__restrict__ idx, int *__restrict__ c20) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = nprob;  // problem of point i: last p with pofs[p] <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pofs[mid] <= i) lo = mid;
    else hi = mid;
  }
  uint64_t c[3] = {0, 0, 0};
  const double m = (double)(1 << MAXD);
  for (int d = 0; d < dim; d++) {
    int64_t v = (int64_t)floor(pts[i * dim + d] * m);
    v = v < 0 ? 0 : (v > (1 << MAXD) - 1 ? (1 << MAXD) - 1 : v);
    c[d] = (uint64_t)v;
    c20[i * dim + d] = (int)v;
  }
  const uint64_t mk = dim == 2 ? (spread2(c[0]) | (spread2(c[1]) << 1))
                               : (spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2));
  mkey[i] = mk;
  key[i] = ((uint64_t)lo << (dim * MAXD)) | mk;
  idx[i] = i;
}

// Radix sort pass, part 1: per block, the counts of the 8-bit digit at
// `shift` over its tile, stored digit-major (digit * nblk + block).
__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint64_t *__restrict__ key, int64_t n, int shift,
                                                  uint32_t *__restrict__ hist, int nblk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_ITEMS; it++) {
    const int64_t e = t0 + it * RS_T + threadIdx.x;
    if (e < n) atomicAdd(&h[(key[e] >> shift) & 255], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// In-place exclusive scan of len counts by one block of 1024 threads, 8192
// consecutive counts at a time (8 per thread, loaded together; warp scans
// of the threads' sums, then the warps' totals), with a running carry.
// total (may be NULL) receives the sum.
template <typename U>
__global__ void __launch_bounds__(1024) k_scan_excl(U *a, int64_t len, U *total) {
  constexpr int IT = 8;
  __shared__ U wsum[32];
  __shared__ U s_carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < len; b0 += 1024 * IT) {
    const int64_t i0 = b0 + (int64_t)tid * IT;
    U v[IT], sum = 0;
#pragma unroll
    for (int u = 0; u < IT; u++) {
      v[u] = i0 + u < len ? a[i0 + u] : (U)0;
      sum += v[u];
    }
    U x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const U y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      U w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const U y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const U carry = s_carry;
    const U incl = x + (warp > 0 ? wsum[warp - 1] : (U)0);
    U run = carry + incl - sum;
#pragma unroll
    for (int u = 0; u < IT; u++) {
      if (i0 + u < len) a[i0 + u] = run;
      run += v[u];
    }
    __syncthreads();
    if (tid == 1023) s_carry = carry + incl;
    __syncthreads();
  }
  if (total && tid == 0) *total = s_carry;
}

// Radix sort pass, part 2: stable scatter.  Each block walks its tile in
// sub-tiles of RS_T keys in index order; a key's position is its digit's
// offset for the block, plus the keys with that digit in earlier sub-tiles,
// earlier warps and earlier lanes of its warp.
__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint64_t *__restrict__ kin, const int64_t *__restrict__ iin,
                                                     uint64_t *__restrict__ kout, int64_t *__restrict__ iout, int64_t n,
                                                     int shift, const uint32_t *__restrict__ offs, int nblk) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[RS_T / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offs[(int64_t)tid * nblk + blockIdx.x];
  const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_ITEMS; it++) {
    for (int d = lane; d < 256; d += 32) wcnt[warp][d] = 0;
    __syncthreads();
    const int64_t e = t0 + it * RS_T + tid;
    const bool ok = e < n;
    const uint64_t k = ok ? kin[e] : 0;
    const int64_t ix = ok ? iin[e] : 0;
    const int dig = ok ? (int)((k >> shift) & 255) : 256 + lane;  // absent keys: a digit of their own
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (ok && rank == 0) wcnt[warp][dig] = __popc(peers);
    __syncthreads();
    if (ok) {
      uint32_t pos = base[dig] + (uint32_t)rank;
      for (int w = 0; w < warp; w++) pos += wcnt[w][dig];
      kout[pos] = k;
      iout[pos] = ix;
    }
    __syncthreads();
    uint32_t s = 0;
    for (int w = 0; w < RS_T / 32; w++) s += wcnt[w][tid];
    base[tid] += s;
    __syncthreads();
  }
}

// First position q in [0, n) with (key[q] >> sh) >= P, and the first with > P.
__device__ __forceinline__ int64_t prefix_lower(const uint64_t *key, int64_t n, uint64_t P, int sh) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((key[mid] >> sh) < P) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int64_t prefix_upper(const uint64_t *key, int64_t n, uint64_t P, int sh) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((key[mid] >> sh) <= P) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// First depth at which sorted point p starts a run (0 for the first point of
// a problem; 21: never, its key equals its predecessor's).
__device__ __forceinline__ int run_start_depth(const uint64_t *key, int64_t p, int dim) {
  if (p == 0) return 0;
  const uint64_t x = key[p] ^ key[p - 1];
  if (x == 0) return MAXD + 1;
  const int hb = 63 - __clzll((long long)x);
  const int t = MAXD - hb / dim;
  return t < 0 ? 0 : t;
}

// Leaf depth of every sorted point, and the number of nodes each starts.
__global__ void k_tree_depths(const uint64_t *__restrict__ key, int64_t n, int dim, int leaf, int *__restrict__ L,
                              uint32_t *__restrict__ nd) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  int lo = 0, hi = MAXD;  // first depth whose run holds <= leaf points, or 20
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int sh = dim * (MAXD - mid);
    const uint64_t P = key[p] >> sh;
    const int64_t cnt = prefix_upper(key, n, P, sh) - prefix_lower(key, n, P, sh);
    if (cnt <= leaf) hi = mid;
    else lo = mid + 1;
  }
  L[p] = lo;
  const int tb = run_start_depth(key, p, dim);
  nd[p] = tb <= lo ? (uint32_t)(lo - tb + 1) : 0u;
}

// The nodes (pre-order ids = exclusive scan of the per-point counts): depth,
// parent, coordinates, first point and count.  Points are sorted positions;
// prob_first (per problem) turns them into positions within the problem.
__global__ void k_tree_nodes(const uint64_t *__restrict__ key, const int *__restrict__ c20s, int64_t n, int dim,
                             const int *__restrict__ L, const uint32_t *__restrict__ base, int *__restrict__ depth,
                             int *__restrict__ parent, int *__restrict__ coord, int64_t *__restrict__ start,
                             int64_t *__restrict__ count) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int tb = run_start_depth(key, p, dim), lp = L[p];
  for (int t = tb; t <= lp; t++) {
    const int id = (int)base[p] + (t - tb);
    const int sh = dim * (MAXD - t);
    depth[id] = t;
    start[id] = p;
    count[id] = prefix_upper(key, n, key[p] >> sh, sh) - p;
    for (int d = 0; d < 3; d++) coord[3 * id + d] = d < dim ? (c20s[p * dim + d] >> (MAXD - t)) : 0;
    if (t > tb) {
      parent[id] = id - 1;  // the parent starts at the same point
    } else if (t == 0) {
      parent[id] = -1;
    } else {
      const int shp = dim * (MAXD - t + 1);
      const int64_t s = prefix_lower(key, n, key[p] >> shp, shp);
      parent[id] = (int)base[s] + (t - 1 - run_start_depth(key, s, dim));
    }
  }
}

// Points of a leaf shallower than 20 back in original order; deeper leaves
// (equal keys) already are, by the stable sort.
__global__ void k_tree_leaf_order(const uint64_t *__restrict__ key, const int64_t *__restrict__ idx, int64_t n,
                                  int dim, const int *__restrict__ L, int64_t *__restrict__ perm) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int lp = L[p];
  if (lp >= MAXD) {
    perm[p] = idx[p];
    return;
  }
  const int sh = dim * (MAXD - lp);
  const uint64_t P = key[p] >> sh;
  const int64_t s = prefix_lower(key, n, P, sh), e = prefix_upper(key, n, P, sh);
  const int64_t me = idx[p];
  int64_t rank = 0;
  for (int64_t q = s; q < e; q++) rank += idx[q] < me;
  perm[s + rank] = me;
}

// Tree-order copies: coordinates, depth-20 cells and Morton keys.
__global__ void k_tree_gather(const double *__restrict__ pts, const int *__restrict__ c20, const uint64_t *__restrict__ mkey,
                              const int64_t *__restrict__ perm, int64_t n, int dim, double *__restrict__ x,
                              int *__restrict__ c20t, uint64_t *__restrict__ keyt) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  const int64_t i = perm[g];
  for (int d = 0; d < dim; d++) {
    x[g * dim + d] = pts[i * dim + d];
    c20t[g * dim + d] = c20[i * dim + d];
  }
  keyt[g] = mkey[i];
}

__global__ void k_tree_sorted_cells(const int *__restrict__ c20, const int64_t *__restrict__ idx, int64_t n, int dim,
                                    int *__restrict__ c20s) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int64_t i = idx[p];
  for (int d = 0; d < dim; d++) c20s[p * dim + d] = c20[i * dim + d];
}

inline unsigned nb256(int64_t n) { return (unsigned)((n + 255) / 256); }


// ---------------------------------------------------------------------------
// Level lists of one problem on the GPU.  The active DOFs of a level (tree
// order, ascending) fall into the depth-t cells of their Morton keys (the
// depth-20 key shifted right by dim (20 - t) bits); the list is sorted by
// key, so a cell is a run of the list.  Its neighbours at Chebyshev
// distance <= 2 (codes 0 .. 5^dim - 1) come from a dense lookup grid of the
// level (side^dim cells), or by binary search in the sorted cell keys when
// that grid would be too large; the pair blocks (cell, neighbour) are laid
// out cell by cell in code order, each b_cell x b_neighbour.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t compact2(uint64_t x) {
  x &= 0x5555555555555555ULL;
  x = (x | (x >> 1)) & 0x3333333333333333ULL;
  x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0fULL;
  x = (x | (x >> 4)) & 0x00ff00ff00ff00ffULL;
  x = (x | (x >> 8)) & 0x0000ffff0000ffffULL;
  x = (x | (x >> 16)) & 0x00000000ffffffffULL;
  return (uint32_t)x;
}
__device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ULL;
  x = (x | (x >> 2)) & 0x10c30c30c30c30c3ULL;
  x = (x | (x >> 4)) & 0x100f00f00f00f00fULL;
  x = (x | (x >> 8)) & 0x001f0000ff0000ffULL;
  x = (x | (x >> 16)) & 0x001f00000000ffffULL;
  x = (x | (x >> 32)) & 0x00000000001fffffULL;
  return (uint32_t)x;
}

// depth-t keys of the active DOFs; *unsorted != 0 when the list is not in
// key order (DOFs of a leaf shallower than t keep their original order)
__global__ void k_lv_keys(const uint64_t *__restrict__ key, const int64_t *__restrict__ act, int64_t na, int ksh,
                          uint64_t *__restrict__ dk, uint32_t *unsorted) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= na) return;
  const uint64_t k = key[act[q]] >> ksh;
  dk[q] = k;
  if (q > 0 && (key[act[q - 1]] >> ksh) > k) atomicOr(unsorted, 1u);
}

// run starts of the key-ordered list
__global__ void k_lv_runs(const uint64_t *__restrict__ dk, int64_t na, uint32_t *__restrict__ flag) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= na) return;
  flag[q] = (q == 0 || dk[q - 1] != dk[q]) ? 1u : 0u;
}

// cpos: exclusive scan of the run starts (the cell of each DOF at a start)
__global__ void k_lv_cells(const int64_t *__restrict__ act, int64_t na, int dim, const uint64_t *__restrict__ dk,
                           const uint32_t *__restrict__ flag, const uint32_t *__restrict__ cpos,
                           int64_t *__restrict__ cell_dof_off, int64_t *__restrict__ cell_dofs,
                           uint64_t *__restrict__ cell_key, int *__restrict__ cell_coord) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= na) return;
  cell_dofs[q] = act[q];
  if (q == na - 1) cell_dof_off[cpos[q] + flag[q]] = na;
  if (!flag[q]) return;
  const uint32_t c = cpos[q];
  const uint64_t k = dk[q];
  cell_dof_off[c] = q;
  cell_key[c] = k;
  if (dim == 2) {
    cell_coord[3 * c] = (int)compact2(k);
    cell_coord[3 * c + 1] = (int)compact2(k >> 1);
    cell_coord[3 * c + 2] = 0;
  } else {
    cell_coord[3 * c] = (int)compact3(k);
    cell_coord[3 * c + 1] = (int)compact3(k >> 1);
    cell_coord[3 * c + 2] = (int)compact3(k >> 2);
  }
}

__global__ void k_lv_sizes(int ncell, const int64_t *__restrict__ cell_dof_off, int *__restrict__ cell_b, int *bmax,
                           int *__restrict__ grid, int side, int dim, const int *__restrict__ cell_coord) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int b = (int)(cell_dof_off[c + 1] - cell_dof_off[c]);
  cell_b[c] = b;
  atomicMax(bmax, b);
  if (grid) {
    int64_t lin = 0, mul = 1;
    for (int d = 0; d < dim; d++) lin += (int64_t)cell_coord[3 * c + d] * mul, mul *= side;
    grid[lin] = c;
  }
}

// cell of integer coordinates p at this level, or -1
__device__ __forceinline__ int lv_lookup(const int64_t *p, int dim, int side, const int *grid,
                                         const uint64_t *cell_key, int ncell) {
  for (int d = 0; d < dim; d++)
    if (p[d] < 0 || p[d] >= side) return -1;
  if (grid) {
    int64_t lin = 0, mul = 1;
    for (int d = 0; d < dim; d++) lin += p[d] * mul, mul *= side;
    return grid[lin];
  }
  const uint64_t k = dim == 2 ? (spread2((uint64_t)p[0]) | (spread2((uint64_t)p[1]) << 1))
                              : (spread3((uint64_t)p[0]) | (spread3((uint64_t)p[1]) << 1) |
                                 (spread3((uint64_t)p[2]) << 2));
  int lo = 0, hi = ncell;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cell_key[mid] < k) lo = mid + 1;
    else hi = mid;
  }
  return lo < ncell && cell_key[lo] == k ? lo : -1;
}

// one thread per (cell, code): the neighbour and the size of the pair block
__global__ void k_lv_nbrs(int ncell, int dim, int NB, int side, const int *__restrict__ grid,
                          const uint64_t *__restrict__ cell_key, const int *__restrict__ cell_coord,
                          const int *__restrict__ cell_b, int *__restrict__ cell_nbr,
                          unsigned long long *__restrict__ psz) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)ncell * NB) return;
  const int c = (int)(e / NB), code = (int)(e % NB);
  const int dx = code % 5 - 2, dy = (code / 5) % 5 - 2, dz = dim == 3 ? code / 25 - 2 : 0;
  const int64_t p[3] = {cell_coord[3 * c] + dx, cell_coord[3 * c + 1] + dy, cell_coord[3 * c + 2] + dz};
  const int nb = lv_lookup(p, dim, side, grid, cell_key, ncell);
  cell_nbr[e] = nb;
  psz[e] = nb >= 0 ? (unsigned long long)cell_b[c] * (unsigned long long)cell_b[nb] : 0ull;
}

__global__ void k_lv_pairoff(int64_t len, const int *__restrict__ cell_nbr, const unsigned long long *__restrict__ excl,
                             int64_t *__restrict__ pair_off) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= len) return;
  pair_off[e] = cell_nbr[e] >= 0 ? (int64_t)excl[e] : -1;
}

// one thread per tree node of depth t: its cell (-1 if none of its DOFs is
// active) and the sizes the factor's records need: b, the DOFs of the cell
// and its near cells, those of its ring cells (distance 2) and the numbers
// of near and ring cells present
__global__ void k_lv_boxes(int nbox, const int *__restrict__ node_coord, int dim, int side, int NB,
                           const int *__restrict__ grid, const uint64_t *__restrict__ cell_key, int ncell,
                           const int *__restrict__ cell_b, const int *__restrict__ cell_nbr,
                           int *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbox) return;
  const int64_t p[3] = {node_coord[3 * i], node_coord[3 * i + 1], node_coord[3 * i + 2]};
  const int c = lv_lookup(p, dim, side, grid, cell_key, ncell);
  int *o = out + 6 * (int64_t)i;
  o[0] = c;
  if (c < 0) return;
  const int b = cell_b[c];
  int nj = b, nnc = 0, ring = 0, nrc = 0;
  for (int code = 0; code < NB; code++) {
    const int dx = code % 5 - 2, dy = (code / 5) % 5 - 2, dz = dim == 3 ? code / 25 - 2 : 0;
    const int dist = max(abs(dx), max(abs(dy), abs(dz)));
    const int nb = cell_nbr[(int64_t)c * NB + code];
    if (nb < 0 || dist == 0) continue;
    if (dist == 1) nj += cell_b[nb], nnc++;
    else ring += cell_b[nb], nrc++;
  }
  o[1] = b;
  o[2] = nj;
  o[3] = ring;
  o[4] = nnc;
  o[5] = nrc;
}

// the next level's active DOFs: each cell's survivors (local indices in
// act_idx, ascending) at the exclusive scan of the counts
__global__ void k_lv_compact(int ncell, const int64_t *__restrict__ cell_dof_off, const int64_t *__restrict__ cell_dofs,
                             const int *__restrict__ act_cnt, const int *__restrict__ act_idx,
                             const uint32_t *__restrict__ aoff, int64_t *__restrict__ next) {
  const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (c >= ncell) return;
  const int64_t o = cell_dof_off[c];
  for (int q = lane; q < act_cnt[c]; q += 32) next[aoff[c] + q] = cell_dofs[o + act_idx[o + q]];
}

}  // namespace

int64_t tree_gpu_scratch_bytes(int64_t n, int dim) {
  const int64_t nblk = (n + RS_TILE - 1) / RS_TILE;
  auto r16 = [](int64_t b) { return (b + 15) & ~(int64_t)15; };
  return 3 * r16(8 * n) + 2 * r16(8 * n) + 2 * r16(4 * n * dim) + 2 * r16(4 * n) + r16(4 * 256 * nblk) + 16 + 64;
}

void tree_gpu_sort(TreeGpu &T, void *scratch, cudaStream_t st) {
  unsigned char *w = static_cast<unsigned char *>(scratch);
  auto take = [&](int64_t bytes) {
    void *r = w;
    w += (bytes + 15) & ~(int64_t)15;
    return r;
  };
  const int64_t n = T.n;
  const int dim = T.dim;
  T.k0 = (uint64_t *)take(8 * n);
  T.k1 = (uint64_t *)take(8 * n);
  T.mkey = (uint64_t *)take(8 * n);
  T.i0 = (int64_t *)take(8 * n);
  T.i1 = (int64_t *)take(8 * n);
  T.c20 = (int *)take(4 * n * dim);
  T.c20s = (int *)take(4 * n * dim);
  T.Lp = (int *)take(4 * n);
  T.nd = (uint32_t *)take(4 * n);
  T.nblk = (n + RS_TILE - 1) / RS_TILE;
  T.hist = (uint32_t *)take(4 * 256 * T.nblk);
  T.total = (uint32_t *)take(16);
  cudaMemsetAsync(T.total, 0, sizeof(uint32_t), st);
  if (n == 0) return;
  k_tree_keys<<<nb256(n), 256, 0, st>>>(T.pts, n, dim, T.pofs, T.nprob, T.k0, T.mkey, T.i0, T.c20); count_launch();
  const int bits = dim * MAXD + T.prob_bits;
  for (int sh = 0; sh < bits; sh += 8) {
    k_rs_hist<<<(unsigned)T.nblk, RS_T, 0, st>>>(T.k0, n, sh, T.hist, (int)T.nblk); count_launch();
    k_scan_excl<uint32_t><<<1, 1024, 0, st>>>(T.hist, 256 * T.nblk, nullptr); count_launch();
    k_rs_scatter<<<(unsigned)T.nblk, RS_T, 0, st>>>(T.k0, T.i0, T.k1, T.i1, n, sh, T.hist, (int)T.nblk);
    count_launch();
    std::swap(T.k0, T.k1);
    std::swap(T.i0, T.i1);
  }
  k_tree_depths<<<nb256(n), 256, 0, st>>>(T.k0, n, dim, T.leaf, T.Lp, T.nd); count_launch();
  k_scan_excl<uint32_t><<<1, 1024, 0, st>>>(T.nd, n, T.total); count_launch();
}

void tree_gpu_nodes(const TreeGpu &T, int *depth, int *parent, int *coord, int64_t *start, int64_t *count,
                    int64_t *perm, double *x, int *c20t, uint64_t *keyt, cudaStream_t st) {
  const int64_t n = T.n;
  if (n == 0) return;
  k_tree_sorted_cells<<<nb256(n), 256, 0, st>>>(T.c20, T.i0, n, T.dim, T.c20s); count_launch();
  k_tree_nodes<<<nb256(n), 256, 0, st>>>(T.k0, T.c20s, n, T.dim, T.Lp, T.nd, depth, parent, coord, start, count);
  count_launch();
  k_tree_leaf_order<<<nb256(n), 256, 0, st>>>(T.k0, T.i0, n, T.dim, T.Lp, perm); count_launch();
  k_tree_gather<<<nb256(n), 256, 0, st>>>(T.pts, T.c20, T.mkey, perm, n, T.dim, x, c20t, keyt); count_launch();
}

// A factor's per-point arrays from the tree-order points: each point's
// depth-20 cell padded to three coordinates, and its offset from the cell's
// corner in FP32 (x - c 2^-20; zero in unused coordinates).
__global__ void k_points_setup(const double *__restrict__ x, const int *__restrict__ c20, int64_t n, int dim,
                               double D, int *__restrict__ cell3, float *__restrict__ off) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const int c = d < dim ? c20[g * dim + d] : 0;
    cell3[3 * g + d] = c;
    off[3 * g + d] = d < dim ? (float)(x[g * dim + d] - (double)c * D) : 0.f;
  }
}

void points_setup(const double *x, const int *c20, int64_t n, int dim, double D, int *cell3, float *off,
                  cudaStream_t st) {
  if (n == 0) return;
  k_points_setup<<<nb256(n), 256, 0, st>>>(x, c20, n, dim, D, cell3, off); count_launch();
}

// Is every point the centre ((i + 1/2) / s) of its own cell of an s^dim
// grid?  Records each point's grid index in caller order; *bad != 0 when a
// coordinate is off the centres or a cell is used twice (seen: n flags,
// zeroed by the caller).
__global__ void k_grid_detect(const double *__restrict__ x, const int64_t *__restrict__ perm, int64_t n, int dim,
                              int64_t s, int64_t *__restrict__ gidx, unsigned *__restrict__ seen, int *bad) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  int64_t lin = 0, mul = 1;
  for (int d = 0; d < dim; d++) {
    const double v = x[g * dim + d] * (double)s - 0.5;
    const double iv = nearbyint(v);
    if (v != iv || iv < 0 || iv >= (double)s) {
      atomicOr(bad, 1);
      return;
    }
    lin += (int64_t)iv * mul;
    mul *= s;
  }
  if (atomicExch(&seen[lin], 1u)) {
    atomicOr(bad, 1);
    return;
  }
  gidx[perm[g]] = lin;
}

void grid_detect(const double *x, const int64_t *perm, int64_t n, int dim, int64_t s, int64_t *gidx, unsigned *seen,
                 int *bad, cudaStream_t st) {
  if (n == 0) return;
  k_grid_detect<<<nb256(n), 256, 0, st>>>(x, perm, n, dim, s, gidx, seen, bad); count_launch();
}


void level_gpu_keys(const uint64_t *key, const int64_t *act, int64_t na, int ksh, uint64_t *dk, uint32_t *unsorted,
                    cudaStream_t st) {
  if (na == 0) return;
  k_lv_keys<<<nb256(na), 256, 0, st>>>(key, act, na, ksh, dk, unsorted); count_launch();
}

void level_gpu_runs(const uint64_t *dk, int64_t na, uint32_t *flag, uint32_t *cpos, uint32_t *ncell, cudaStream_t st) {
  if (na == 0) return;
  k_lv_runs<<<nb256(na), 256, 0, st>>>(dk, na, flag); count_launch();
  cudaMemcpyAsync(cpos, flag, sizeof(uint32_t) * (size_t)na, cudaMemcpyDeviceToDevice, st);
  k_scan_excl<uint32_t><<<1, 1024, 0, st>>>(cpos, na, ncell); count_launch();
}

int64_t sort_pairs_hist_bytes(int64_t n) { return 4 * 256 * ((n + RS_TILE - 1) / RS_TILE) + 16; }

void sort_pairs_u64(uint64_t *k0, int64_t *v0, uint64_t *k1, int64_t *v1, uint32_t *hist, int64_t n, int bits,
                    cudaStream_t st) {
  if (n <= 1) return;
  const int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
  uint64_t *ka = k0, *kb = k1;
  int64_t *va = v0, *vb = v1;
  for (int sh = 0; sh < bits; sh += 8) {
    k_rs_hist<<<(unsigned)nblk, RS_T, 0, st>>>(ka, n, sh, hist, nblk); count_launch();
    k_scan_excl<uint32_t><<<1, 1024, 0, st>>>(hist, 256 * (int64_t)nblk, nullptr); count_launch();
    k_rs_scatter<<<(unsigned)nblk, RS_T, 0, st>>>(ka, va, kb, vb, n, sh, hist, nblk); count_launch();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != k0) {
    cudaMemcpyAsync(k0, ka, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(v0, va, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
  }
}

void level_gpu_tables(const LevelGpu &L, cudaStream_t st) {
  if (L.na == 0 || L.ncell == 0) return;
  k_lv_cells<<<nb256(L.na), 256, 0, st>>>(L.act, L.na, L.dim, L.dk, L.flag, L.cpos, L.cell_dof_off, L.cell_dofs,
                                          L.cell_key, L.cell_coord);
  count_launch();
  k_lv_sizes<<<nb256(L.ncell), 256, 0, st>>>(L.ncell, L.cell_dof_off, L.cell_b, L.bmax, L.grid, L.side, L.dim,
                                             L.cell_coord);
  count_launch();
  const int64_t len = (int64_t)L.ncell * L.NB;
  k_lv_nbrs<<<nb256(len), 256, 0, st>>>(L.ncell, L.dim, L.NB, L.side, L.grid, L.cell_key, L.cell_coord, L.cell_b,
                                        L.cell_nbr, L.psz);
  count_launch();
  k_scan_excl<unsigned long long><<<1, 1024, 0, st>>>(L.psz, len, L.pool_total); count_launch();
  k_lv_pairoff<<<nb256(len), 256, 0, st>>>(len, L.cell_nbr, L.psz, L.pair_off); count_launch();
  if (L.nbox > 0) {
    k_lv_boxes<<<nb256(L.nbox), 256, 0, st>>>(L.nbox, L.node_coord, L.dim, L.side, L.NB, L.grid, L.cell_key, L.ncell,
                                              L.cell_b, L.cell_nbr, L.box_out);
    count_launch();
  }
}

void level_gpu_next_active(int ncell, const int64_t *cell_dof_off, const int64_t *cell_dofs, const int *act_cnt,
                           const int *act_idx, uint32_t *aoff, uint32_t *total, int64_t *next, cudaStream_t st) {
  if (ncell == 0) return;
  cudaMemcpyAsync(aoff, act_cnt, sizeof(uint32_t) * (size_t)ncell, cudaMemcpyDeviceToDevice, st);
  k_scan_excl<uint32_t><<<1, 1024, 0, st>>>(aoff, ncell, total); count_launch();
  k_lv_compact<<<(unsigned)(((int64_t)ncell * 32 + 255) / 256), 256, 0, st>>>(ncell, cell_dof_off, cell_dofs, act_cnt,
                                                                            act_idx, aoff, next);
  count_launch();
}

__global__ void k_iota64(int64_t *p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}
void iota64(int64_t *p, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  k_iota64<<<nb256(n), 256, 0, st>>>(p, n); count_launch();
}

}  // namespace rss
