// api.cu -- host orchestration and the C ABI (include/rss.h).
//
// The factorization follows Algorithm 1 of the paper: levels (tree depths)
// from the finest to depth 2, boxes of a level in colour-major order.  All
// arithmetic runs in the kernels of kernels.cu; the host builds the index
// structures of each level (which cells hold active DOFs, their neighbour
// tables and pair-block offsets) once the ranks of the previous level are
// known, and launches one ID / elimination / Schur launch per colour phase.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/rss.h"
#include "internal.h"

namespace rss {

static thread_local std::string g_last_error;

struct Fail {
  rss_status st;
  std::string msg;
};

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      cudaGetLastError();                                                              \
      throw Fail{e_ == cudaErrorMemoryAllocation ? RSS_ENOMEM : RSS_ECUDA,             \
                 std::string(#call) + ": " + cudaGetErrorString(e_)};                  \
    }                                                                                  \
  } while (0)

static void check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Fail{RSS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

// ---------------------------------------------------------------------------
// Device memory: one library-private stream-ordered pool.
// ---------------------------------------------------------------------------

static cudaMemPool_t lib_pool() {
  static cudaMemPool_t pool = nullptr;
  static int dev_of_pool = -1;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (!pool || dev_of_pool != dev) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    CK(cudaMemPoolCreate(&pool, &props));
    uint64_t thr = UINT64_MAX;
    CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    dev_of_pool = dev;
  }
  return pool;
}

struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  ~DBuf() { release(); }
  void alloc(size_t nb, cudaStream_t s) {
    release();
    st = s;
    bytes = nb;
    if (nb == 0) nb = 16;
    CK(cudaMallocFromPoolAsync(&p, nb, lib_pool(), s));
  }
  void release() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    bytes = 0;
  }
};

template <typename U> static inline U *ptr(const DBuf &b) { return static_cast<U *>(b.p); }

template <typename U> static void upload(DBuf &d, const std::vector<U> &h, cudaStream_t st) {
  d.alloc(h.size() * sizeof(U), st);
  if (!h.empty()) CK(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(U), cudaMemcpyHostToDevice, st));
}

// ---------------------------------------------------------------------------
// Tree
// ---------------------------------------------------------------------------

static const uint32_t MAGIC_TREE = 0x52535354u, MAGIC_FACTOR = 0x52535346u;

static inline int64_t cell_at(double v, int t) {
  int64_t m = (int64_t)1 << t;
  int64_t c = (int64_t)floor(v * (double)m);
  return c < 0 ? 0 : (c > m - 1 ? m - 1 : c);
}

static inline uint64_t morton_key(const int64_t *c, int dim, int bits) {
  uint64_t k = 0;
  for (int b = 0; b < bits; b++)
    for (int d = 0; d < dim; d++) k |= (uint64_t)((c[d] >> b) & 1) << (dim * b + d);
  return k;
}

struct HTree {
  uint32_t magic = MAGIC_TREE;
  int dim = 2, leaf = 64, maxdepth = 0;
  int64_t n = 0;
  std::vector<int64_t> perm;
  std::vector<double> x;  // tree order
  std::vector<int> depth, parent, coord;
  std::vector<int64_t> start, count;
  std::vector<std::vector<int>> level;  // boxes per depth, elimination order
};

static int colour_of(const int *c, int dim) {
  int col = 0, mul = 1;
  for (int d = 0; d < dim; d++) {
    col += (c[d] % 3) * mul;
    mul *= 3;
  }
  return col;
}

// Build by sorting on the depth-20 Morton key: a node of depth t is the run
// of points sharing the key's top dim*t bits; children come out in child
// index order because x is the lowest bit of each group.
static void build_tree(HTree &T, const double *pts_host) {
  const int dim = T.dim;
  const int64_t n = T.n;
  const int MAXD = 20;
  std::vector<uint64_t> key(n);
  for (int64_t i = 0; i < n; i++) {
    int64_t c[3] = {0, 0, 0};
    for (int d = 0; d < dim; d++) c[d] = cell_at(pts_host[i * dim + d], MAXD);
    key[i] = morton_key(c, dim, MAXD);
  }
  T.perm.resize(n);
  for (int64_t i = 0; i < n; i++) T.perm[i] = i;
  std::stable_sort(T.perm.begin(), T.perm.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  std::vector<uint64_t> ks(n);
  for (int64_t g = 0; g < n; g++) ks[g] = key[T.perm[g]];
  T.maxdepth = 0;
  struct Frame {
    int64_t lo, hi;
    int depth, parent;
    int c[3];
  };
  std::vector<Frame> stack;
  stack.push_back({0, n, 0, -1, {0, 0, 0}});
  while (!stack.empty()) {
    Frame f = stack.back();
    stack.pop_back();
    int id = (int)T.depth.size();
    T.depth.push_back(f.depth);
    T.parent.push_back(f.parent);
    for (int d = 0; d < 3; d++) T.coord.push_back(f.c[d]);
    T.start.push_back(f.lo);
    T.count.push_back(f.hi - f.lo);
    T.maxdepth = std::max(T.maxdepth, f.depth);
    if (f.hi - f.lo > T.leaf && f.depth < MAXD) {
      // children: split [lo,hi) by the dim bits of depth f.depth+1
      int shift = dim * (MAXD - f.depth - 1);
      std::vector<Frame> ch;
      int64_t p = f.lo;
      while (p < f.hi) {
        uint64_t grp = (ks[p] >> shift) & ((1u << dim) - 1);
        int64_t q = p;
        while (q < f.hi && ((ks[q] >> shift) & ((1u << dim) - 1)) == grp) q++;
        Frame cf{p, q, f.depth + 1, id, {0, 0, 0}};
        for (int d = 0; d < dim; d++) cf.c[d] = 2 * f.c[d] + (int)((grp >> d) & 1);
        ch.push_back(cf);
        p = q;
      }
      for (int i = (int)ch.size() - 1; i >= 0; i--) stack.push_back(ch[i]);  // pre-order
    } else {
      // a leaf keeps its points in original order
      std::sort(T.perm.begin() + f.lo, T.perm.begin() + f.hi);
    }
  }
  T.x.resize((size_t)n * dim);
  for (int64_t g = 0; g < n; g++)
    for (int d = 0; d < dim; d++) T.x[g * dim + d] = pts_host[T.perm[g] * dim + d];
  T.level.assign(T.maxdepth + 1, {});
  for (int i = 0; i < (int)T.depth.size(); i++) T.level[T.depth[i]].push_back(i);
  for (auto &lv : T.level) {
    std::sort(lv.begin(), lv.end(), [&](int a, int b) {
      int ca = colour_of(&T.coord[3 * a], dim), cb = colour_of(&T.coord[3 * b], dim);
      if (ca != cb) return ca < cb;
      int64_t pa[3] = {T.coord[3 * a], T.coord[3 * a + 1], T.coord[3 * a + 2]};
      int64_t pb[3] = {T.coord[3 * b], T.coord[3 * b + 1], T.coord[3 * b + 2]};
      return morton_key(pa, dim, 21) < morton_key(pb, dim, 21);
    });
  }
}

}  // namespace rss

struct rss_tree {
  uint32_t magic = rss::MAGIC_TREE;
  rss::HTree t;
};

namespace rss {

// ---------------------------------------------------------------------------
// Levels
// ---------------------------------------------------------------------------

struct HLevel {
  int t = 0, ncell = 0, NB = 25, dim = 2;
  std::vector<uint64_t> key;  // sorted cell keys
  std::vector<int> cell_b, cell_coord, cell_nbr;
  std::vector<int64_t> cell_dof_off, cell_dofs, pair_off;
  int64_t pool_elems = 0;
  std::vector<int> box_cell, box_node, box_colour;
  int bmax = 0;
};

template <typename T> struct DLevel {
  DBuf cell_b, cell_dof_off, cell_dofs, cell_coord, cell_nbr, pair_off, act_cnt, act_idx, pool;
  LevelDev<T> view(const HLevel &h, const int *dof_cell, const int *dof_loc) const {
    LevelDev<T> v{};
    v.t = h.t;
    v.dim = h.dim;
    v.ncell = h.ncell;
    v.NB = h.NB;
    v.cell_b = ptr<int>(cell_b);
    v.cell_dof_off = ptr<int64_t>(cell_dof_off);
    v.cell_dofs = ptr<int64_t>(cell_dofs);
    v.cell_coord = ptr<int>(cell_coord);
    v.cell_nbr = ptr<int>(cell_nbr);
    v.pair_off = ptr<int64_t>(pair_off);
    v.act_cnt = ptr<int>(act_cnt);
    v.act_idx = ptr<int>(act_idx);
    v.dof_cell = dof_cell;
    v.dof_loc = dof_loc;
    v.pool = ptr<T>(pool);
    return v;
  }
};

static int find_key(const std::vector<uint64_t> &keys, uint64_t k) {
  auto it = std::lower_bound(keys.begin(), keys.end(), k);
  if (it == keys.end() || *it != k) return -1;
  return (int)(it - keys.begin());
}

static HLevel build_level(const HTree &T, int t, const std::vector<int64_t> &active) {
  HLevel L;
  L.t = t;
  L.dim = T.dim;
  const int dim = T.dim;
  L.NB = dim == 2 ? 25 : 125;
  const int bits = std::max(t, 1);
  std::vector<uint64_t> dk(active.size());
  for (size_t q = 0; q < active.size(); q++) {
    int64_t c[3] = {0, 0, 0};
    for (int d = 0; d < dim; d++) c[d] = cell_at(T.x[active[q] * dim + d], t);
    dk[q] = morton_key(c, dim, bits);
  }
  L.key = dk;
  std::sort(L.key.begin(), L.key.end());
  L.key.erase(std::unique(L.key.begin(), L.key.end()), L.key.end());
  L.ncell = (int)L.key.size();
  L.cell_b.assign(L.ncell, 0);
  std::vector<int> cid(active.size());
  for (size_t q = 0; q < active.size(); q++) {
    cid[q] = find_key(L.key, dk[q]);
    L.cell_b[cid[q]]++;
  }
  L.cell_dof_off.assign(L.ncell + 1, 0);
  for (int c = 0; c < L.ncell; c++) L.cell_dof_off[c + 1] = L.cell_dof_off[c] + L.cell_b[c];
  L.cell_dofs.resize(active.size());
  std::vector<int64_t> fill(L.cell_dof_off.begin(), L.cell_dof_off.end() - 1);
  for (size_t q = 0; q < active.size(); q++) L.cell_dofs[fill[cid[q]]++] = active[q];
  L.cell_coord.assign(3 * L.ncell, 0);
  for (int c = 0; c < L.ncell; c++) {
    uint64_t k = L.key[c];
    for (int d = 0; d < dim; d++) {
      int v = 0;
      for (int b = 0; b < bits; b++) v |= (int)((k >> (dim * b + d)) & 1) << b;
      L.cell_coord[3 * c + d] = v;
    }
  }
  L.cell_nbr.assign((size_t)L.ncell * L.NB, -1);
  L.pair_off.assign((size_t)L.ncell * L.NB, -1);
  const int64_t side = (int64_t)1 << t;
  int64_t off = 0;
  for (int c = 0; c < L.ncell; c++) {
    L.bmax = std::max(L.bmax, L.cell_b[c]);
    int lim = dim == 3 ? 2 : 0;
    for (int dz = -lim; dz <= lim; dz++)
      for (int dy = -2; dy <= 2; dy++)
        for (int dx = -2; dx <= 2; dx++) {
          int64_t p[3] = {L.cell_coord[3 * c] + dx, L.cell_coord[3 * c + 1] + dy, L.cell_coord[3 * c + 2] + dz};
          bool ok = true;
          for (int d = 0; d < dim; d++) ok = ok && p[d] >= 0 && p[d] < side;
          if (!ok) continue;
          int nb = find_key(L.key, morton_key(p, dim, bits));
          if (nb < 0) continue;
          int code = code5(dx, dy, dz, dim);
          L.cell_nbr[(size_t)c * L.NB + code] = nb;
          L.pair_off[(size_t)c * L.NB + code] = off;
          off += (int64_t)L.cell_b[c] * L.cell_b[nb];
        }
  }
  L.pool_elems = off;
  for (int node : T.level[t]) {
    int64_t p[3] = {T.coord[3 * node], T.coord[3 * node + 1], T.coord[3 * node + 2]};
    int c = find_key(L.key, morton_key(p, dim, bits));
    if (c < 0) continue;  // every DOF of the box has become inactive
    L.box_cell.push_back(c);
    L.box_node.push_back(node);
    L.box_colour.push_back(colour_of(&T.coord[3 * node], dim));
  }
  return L;
}

// ---------------------------------------------------------------------------
// Factor
// ---------------------------------------------------------------------------

struct Phase {
  int first, count, bmax;
};

struct FactorBase {
  uint32_t magic = MAGIC_FACTOR;
  int prec = 0;
  virtual ~FactorBase() {}
};

template <typename T> struct Factor : FactorBase {
  HTree tree;
  KernelParams K{};
  ProxyParams px{};
  double eps = 0;
  cudaStream_t st = nullptr;
  int64_t n = 0;
  int dim = 2;
  DBuf d_x, d_perm, d_cell, d_off, d_err;
  Points P{};
  std::vector<std::unique_ptr<DBuf>> store;  // factor storage chunks
  int64_t factor_bytes = 0;
  DBuf d_boxes;
  std::vector<FBox<T>> h_boxes;
  std::vector<Phase> phases;
  int ntop = 0;
  DBuf d_top, d_topLU, d_toppiv;
  mutable DBuf d_work, d_topwork;
  mutable int work_nrhs = 0;

  void *alloc_store(size_t bytes) {
    store.emplace_back(new DBuf());
    store.back()->alloc(bytes, st);
    factor_bytes += (int64_t)bytes;
    return store.back()->p;
  }
};

template <typename T> static void ensure_work(const Factor<T> &F, int nrhs) {
  if (F.work_nrhs >= nrhs) return;
  F.d_work.alloc((size_t)std::max<int64_t>(F.n, 1) * nrhs * sizeof(T), F.st);
  F.d_topwork.alloc((size_t)std::max(F.ntop, 1) * 2 * nrhs * sizeof(T), F.st);
  F.work_nrhs = nrhs;
}

static int check_err(DBuf &d_err, cudaStream_t st) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return h;
}

template <typename T> static void run_factor(Factor<T> &F) {
  HTree &T_ = F.tree;
  const int dim = T_.dim;
  const int64_t n = T_.n;
  cudaStream_t st = F.st;
  // points
  upload(F.d_x, T_.x, st);
  upload(F.d_perm, T_.perm, st);
  {
    int fine = T_.maxdepth;
    double D = ldexp(1.0, -fine);
    std::vector<int> cell((size_t)3 * std::max<int64_t>(n, 1), 0);
    std::vector<float> off((size_t)3 * std::max<int64_t>(n, 1), 0.f);
    for (int64_t g = 0; g < n; g++)
      for (int d = 0; d < dim; d++) {
        int64_t c = cell_at(T_.x[g * dim + d], fine);
        cell[3 * g + d] = (int)c;
        off[3 * g + d] = (float)(T_.x[g * dim + d] - (double)c * D);
      }
    upload(F.d_cell, cell, st);
    upload(F.d_off, off, st);
    F.P.x = ptr<double>(F.d_x);
    F.P.cell = ptr<int>(F.d_cell);
    F.P.off = ptr<float>(F.d_off);
    F.P.D = (float)D;
    F.P.dim = dim;
  }
  F.d_err.alloc(sizeof(int), st);
  CK(cudaMemsetAsync(F.d_err.p, 0, sizeof(int), st));

  int nbox_total = 0;
  for (int t = 2; t <= T_.maxdepth; t++) nbox_total += (int)T_.level[t].size();
  F.d_boxes.alloc(sizeof(FBox<T>) * std::max(nbox_total, 1), st);
  F.h_boxes.clear();
  F.phases.clear();

  std::vector<int64_t> active(n);
  for (int64_t g = 0; g < n; g++) active[g] = g;
  DBuf d_dof_cell[2], d_dof_loc[2];
  std::unique_ptr<DLevel<T>> prevD;
  HLevel prevH;
  int prev_slot = 0;
  bool have_prev = false;

  auto assemble_pairs = [&](const HLevel &H, DLevel<T> &D, const LevelDev<T> *prev) {
    std::vector<int64_t> row_off, col_off, out_off;
    std::vector<int> nrow, ncol;
    int64_t maxblk = 0;
    for (int c = 0; c < H.ncell; c++)
      for (int o = 0; o < H.NB; o++) {
        int nb = H.cell_nbr[(size_t)c * H.NB + o];
        if (nb < 0) continue;
        row_off.push_back(H.cell_dof_off[c]);
        col_off.push_back(H.cell_dof_off[nb]);
        out_off.push_back(H.pair_off[(size_t)c * H.NB + o]);
        nrow.push_back(H.cell_b[c]);
        ncol.push_back(H.cell_b[nb]);
        maxblk = std::max(maxblk, (int64_t)H.cell_b[c] * H.cell_b[nb]);
      }
    DBuf a, b2, c2, d2, e2;
    upload(a, row_off, st);
    upload(b2, col_off, st);
    upload(c2, out_off, st);
    upload(d2, nrow, st);
    upload(e2, ncol, st);
    AssembleList L{(int)row_off.size(), ptr<int64_t>(a), ptr<int64_t>(b2), ptr<int64_t>(c2),
                   ptr<int>(d2), ptr<int>(e2), ptr<int64_t>(D.cell_dofs), ptr<int64_t>(D.cell_dofs), 0};
    launch_assemble<T>(L, ptr<T>(D.pool), prev, F.P, F.K, maxblk, st);
    check_launch("assemble");
  };

  for (int t = T_.maxdepth; t >= 2; t--) {
    HLevel H = build_level(T_, t, active);
    std::unique_ptr<DLevel<T>> D(new DLevel<T>());
    upload(D->cell_b, H.cell_b, st);
    upload(D->cell_dof_off, H.cell_dof_off, st);
    upload(D->cell_dofs, H.cell_dofs, st);
    upload(D->cell_coord, H.cell_coord, st);
    upload(D->cell_nbr, H.cell_nbr, st);
    upload(D->pair_off, H.pair_off, st);
    {
      std::vector<int> ac(H.cell_b), ai(H.cell_dofs.size());
      for (int c = 0; c < H.ncell; c++)
        for (int q = 0; q < H.cell_b[c]; q++) ai[H.cell_dof_off[c] + q] = q;
      upload(D->act_cnt, ac, st);
      upload(D->act_idx, ai, st);
    }
    D->pool.alloc((size_t)H.pool_elems * sizeof(T), st);
    // per-DOF maps of this level
    int slot = have_prev ? 1 - prev_slot : 0;
    {
      std::vector<int> dc(std::max<int64_t>(n, 1), -1), dl(std::max<int64_t>(n, 1), -1);
      for (int c = 0; c < H.ncell; c++)
        for (int q = 0; q < H.cell_b[c]; q++) {
          int64_t g = H.cell_dofs[H.cell_dof_off[c] + q];
          dc[g] = c;
          dl[g] = q;
        }
      upload(d_dof_cell[slot], dc, st);
      upload(d_dof_loc[slot], dl, st);
    }
    LevelDev<T> view = D->view(H, ptr<int>(d_dof_cell[slot]), ptr<int>(d_dof_loc[slot]));
    if (have_prev) {
      LevelDev<T> pv = prevD->view(prevH, ptr<int>(d_dof_cell[prev_slot]), ptr<int>(d_dof_loc[prev_slot]));
      assemble_pairs(H, *D, &pv);
    } else {
      assemble_pairs(H, *D, nullptr);
    }
    prevD.reset();  // stream-ordered free of the previous level

    // factor records of this level's boxes
    const int base = (int)F.h_boxes.size();
    const int nb = (int)H.box_cell.size();
    int njmax_lvl = 0;
    std::vector<int> njmaxv(nb);
    size_t sz_i64 = 0, sz_i32 = 0, sz_T = 0;
    for (int q = 0; q < nb; q++) {
      int c = H.box_cell[q], b = H.cell_b[c];
      int nj = b;
      int lim = dim == 3 ? 1 : 0;
      for (int dz = -lim; dz <= lim; dz++)
        for (int dy = -1; dy <= 1; dy++)
          for (int dx = -1; dx <= 1; dx++) {
            if (!dx && !dy && !dz) continue;
            int nbc = H.cell_nbr[(size_t)c * H.NB + code5(dx, dy, dz, dim)];
            if (nbc >= 0) nj += H.cell_b[nbc];
          }
      njmaxv[q] = nj;
      njmax_lvl = std::max(njmax_lvl, nj);
      sz_i64 += (size_t)b + nj;
      sz_i32 += (size_t)b + 2 * (size_t)nj + b;
      sz_T += (size_t)b * b / 4 + 1 + (size_t)b * b + 2 * (size_t)nj * b;
    }
    int64_t *p64 = (int64_t *)F.alloc_store(sz_i64 * sizeof(int64_t));
    int *p32 = (int *)F.alloc_store(sz_i32 * sizeof(int));
    T *pT = (T *)F.alloc_store(sz_T * sizeof(T));
    for (int q = 0; q < nb; q++) {
      int c = H.box_cell[q], b = H.cell_b[c], nj = njmaxv[q];
      FBox<T> fb{};
      fb.cell = c;
      fb.depth = t;
      fb.b = b;
      fb.njmax = nj;
      fb.ids = p64;
      p64 += b;
      fb.J = p64;
      p64 += nj;
      fb.loc = p32;
      p32 += b;
      fb.Jnb = p32;
      p32 += nj;
      fb.Jloc = p32;
      p32 += nj;
      fb.piv = p32;
      p32 += b;
      fb.Tm = pT;
      pT += (size_t)b * b / 4 + 1;
      fb.LU = pT;
      pT += (size_t)b * b;
      fb.E = pT;
      pT += (size_t)nj * b;
      fb.G = pT;
      pT += (size_t)nj * b;
      F.h_boxes.push_back(fb);
    }
    CK(cudaMemcpyAsync(ptr<FBox<T>>(F.d_boxes) + base, F.h_boxes.data() + base, sizeof(FBox<T>) * nb,
                       cudaMemcpyHostToDevice, st));
    // colour phases
    std::vector<int> list(nb);
    for (int q = 0; q < nb; q++) list[q] = base + q;
    DBuf d_list;
    upload(d_list, list, st);
    int maxphase = 0;
    std::vector<std::pair<int, int>> ph;
    for (int q = 0; q < nb;) {
      int q2 = q;
      while (q2 < nb && H.box_colour[q2] == H.box_colour[q]) q2++;
      ph.push_back({q, q2 - q});
      maxphase = std::max(maxphase, q2 - q);
      q = q2;
    }
    // scratch
    int PR = H.bmax <= 80 ? 128 : 64;
    int64_t idb = id_region_bytes<T>(H.bmax, PR);
    bool id_smem = idb <= 200 * 1024;
    DBuf gid, gel;
    int64_t id_stride = (idb + sizeof(T) - 1) / sizeof(T) + 32;
    if (!id_smem) gid.alloc((size_t)id_stride * sizeof(T) * std::max(maxphase, 1), st);
    int64_t el_stride = 2 * (int64_t)njmax_lvl * H.bmax + 32;
    gel.alloc((size_t)el_stride * sizeof(T) * std::max(maxphase, 1), st);
    for (auto &p : ph) {
      const int *bl = ptr<int>(d_list) + p.first;
      launch_id<T>(view, ptr<FBox<T>>(F.d_boxes), bl, p.second, H.bmax, 0, F.P, F.K, F.px, F.eps,
                   ptr<T>(gid), id_stride, id_smem, st, ptr<int>(F.d_err));
      check_launch("id");
      launch_elim<T>(view, ptr<FBox<T>>(F.d_boxes), bl, p.second, H.bmax, ptr<T>(gel), el_stride, st,
                     ptr<int>(F.d_err));
      check_launch("elim");
      launch_schur<T>(view, ptr<FBox<T>>(F.d_boxes), bl, p.second, njmax_lvl, ptr<T>(gel), el_stride, st);
      check_launch("schur");
      F.phases.push_back({base + p.first, p.second, H.bmax});
    }
    // ranks of this level -> active DOFs of the next
    CK(cudaMemcpyAsync(F.h_boxes.data() + base, ptr<FBox<T>>(F.d_boxes) + base, sizeof(FBox<T>) * nb,
                       cudaMemcpyDeviceToHost, st));
    std::vector<int> ac(H.ncell), ai(H.cell_dofs.size());
    CK(cudaMemcpyAsync(ac.data(), D->act_cnt.p, sizeof(int) * H.ncell, cudaMemcpyDeviceToHost, st));
    if (!ai.empty())
      CK(cudaMemcpyAsync(ai.data(), D->act_idx.p, sizeof(int) * ai.size(), cudaMemcpyDeviceToHost, st));
    int e = check_err(F.d_err, st);
    if (e == DERR_NUMERIC) throw Fail{RSS_ENUMERIC, "zero pivot in the LU of a redundant block"};
    if (e) throw Fail{RSS_ECUDA, "device-side consistency check failed"};
    active.clear();
    for (int c = 0; c < H.ncell; c++)
      for (int q = 0; q < ac[c]; q++) active.push_back(H.cell_dofs[H.cell_dof_off[c] + ai[H.cell_dof_off[c] + q]]);
    std::sort(active.begin(), active.end());
    prevD = std::move(D);
    prevH = std::move(H);
    prev_slot = slot;
    have_prev = true;
  }

  // top block: all DOFs still active (Sec. 3.3.3), dense LU
  F.ntop = (int)active.size();
  upload(F.d_top, active, st);
  F.d_topLU.alloc((size_t)F.ntop * F.ntop * sizeof(T) + 16, st);
  F.d_toppiv.alloc((size_t)F.ntop * sizeof(int) + 16, st);
  F.factor_bytes += (int64_t)F.ntop * F.ntop * sizeof(T) + (int64_t)F.ntop * (sizeof(int) + 8);
  if (F.ntop > 0) {
    std::vector<int64_t> z1{0}, z2{0}, z3{0};
    std::vector<int> nr{F.ntop}, nc{F.ntop};
    DBuf a, b2, c2, d2, e2;
    upload(a, z1, st);
    upload(b2, z2, st);
    upload(c2, z3, st);
    upload(d2, nr, st);
    upload(e2, nc, st);
    AssembleList L{1, ptr<int64_t>(a), ptr<int64_t>(b2), ptr<int64_t>(c2), ptr<int>(d2), ptr<int>(e2),
                   ptr<int64_t>(F.d_top), ptr<int64_t>(F.d_top), 0};
    // the dense LU works on a row-major matrix: assemble the transpose layout
    L.transpose = 1;
    if (have_prev) {
      LevelDev<T> pv = prevD->view(prevH, ptr<int>(d_dof_cell[prev_slot]), ptr<int>(d_dof_loc[prev_slot]));
      launch_assemble<T>(L, ptr<T>(F.d_topLU), &pv, F.P, F.K, (int64_t)F.ntop * F.ntop, st);
    } else {
      launch_assemble<T>(L, ptr<T>(F.d_topLU), nullptr, F.P, F.K, (int64_t)F.ntop * F.ntop, st);
    }
    check_launch("assemble top");
    launch_dense_lu<T>(ptr<T>(F.d_topLU), F.ntop, ptr<int>(F.d_toppiv), st, ptr<int>(F.d_err));
    check_launch("top lu");
  }
  prevD.reset();
  int e = check_err(F.d_err, st);
  if (e == DERR_NUMERIC) throw Fail{RSS_ENUMERIC, "zero pivot in the top block"};
  if (e) throw Fail{RSS_ECUDA, "device-side consistency check failed"};
}

}  // namespace rss

struct rss_factorization {
  uint32_t magic = rss::MAGIC_FACTOR;
  std::unique_ptr<rss::FactorBase> impl;
};

using namespace rss;

template <typename F> static rss_status guard(F &&fn) {
  try {
    fn();
    return RSS_OK;
  } catch (const Fail &f) {
    g_last_error = f.msg;
    return f.st;
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return RSS_ENOMEM;
  } catch (...) {
    g_last_error = "unexpected internal error";
    return RSS_ECUDA;
  }
}

static void fetch_points(const double *pts, int64_t n, int dim, std::vector<double> &h, cudaStream_t st) {
  h.resize((size_t)std::max<int64_t>(n, 1) * dim);
  if (n > 0) {
    CK(cudaMemcpyAsync(h.data(), pts, sizeof(double) * n * dim, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
}

template <typename T> static void do_sweeps(const Factor<T> &F, const double *in, double *out, int nrhs, bool solve) {
  cudaStream_t st = F.st;
  ensure_work(F, nrhs);
  T *v = ptr<T>(F.d_work);
  launch_permute<T>(0, ptr<int64_t>(F.d_perm), in, v, nullptr, F.n, nrhs, st);
  const FBox<T> *bx = ptr<FBox<T>>(F.d_boxes);
  if (solve) {
    for (const Phase &p : F.phases) launch_sweep<T>(SWEEP_SOLVE_FWD, bx, p.first, p.count, v, nrhs, p.bmax, st);
    launch_top<T>(0, ptr<T>(F.d_topLU), ptr<int>(F.d_toppiv), ptr<int64_t>(F.d_top), F.ntop, v, nrhs,
                  ptr<T>(F.d_topwork), st);
    for (auto it = F.phases.rbegin(); it != F.phases.rend(); ++it)
      launch_sweep<T>(SWEEP_SOLVE_BWD, bx, it->first, it->count, v, nrhs, it->bmax, st);
  } else {
    for (const Phase &p : F.phases) launch_sweep<T>(SWEEP_APPLY_FWD, bx, p.first, p.count, v, nrhs, p.bmax, st);
    launch_top<T>(1, ptr<T>(F.d_topLU), ptr<int>(F.d_toppiv), ptr<int64_t>(F.d_top), F.ntop, v, nrhs,
                  ptr<T>(F.d_topwork), st);
    for (auto it = F.phases.rbegin(); it != F.phases.rend(); ++it)
      launch_sweep<T>(SWEEP_APPLY_BWD, bx, it->first, it->count, v, nrhs, it->bmax, st);
  }
  launch_permute<T>(1, ptr<int64_t>(F.d_perm), nullptr, v, out, F.n, nrhs, st);
  check_launch("sweeps");
  CK(cudaStreamSynchronize(st));
}

static rss_status sweep_entry(const rss_factorization *f, const double *in, double *out, int nrhs, bool solve) {
  return guard([&] {
    if (!f || !f->impl || nrhs < 1) throw Fail{RSS_EINVAL, "bad arguments"};
    if (f->impl->prec == RSS_FP64) {
      auto &F = static_cast<const Factor<double> &>(*f->impl);
      if (F.n > 0 && (!in || !out)) throw Fail{RSS_EINVAL, "NULL vector"};
      do_sweeps(F, in, out, nrhs, solve);
    } else {
      auto &F = static_cast<const Factor<float> &>(*f->impl);
      if (F.n > 0 && (!in || !out)) throw Fail{RSS_EINVAL, "NULL vector"};
      do_sweeps(F, in, out, nrhs, solve);
    }
  });
}

extern "C" {

const char *rss_last_error(void) { return g_last_error.c_str(); }

rss_status rss_build_tree(const double *pts, int64_t n, int dim, int leaf_size, rss_tree **out) {
  return guard([&] {
    if (!out || n < 0 || (dim != 2 && dim != 3) || leaf_size < 1 || (n > 0 && !pts))
      throw Fail{RSS_EINVAL, "rss_build_tree: bad arguments"};
    std::unique_ptr<rss_tree> tr(new rss_tree());
    tr->t.dim = dim;
    tr->t.leaf = leaf_size;
    tr->t.n = n;
    std::vector<double> h;
    fetch_points(pts, n, dim, h, nullptr);
    build_tree(tr->t, h.data());
    *out = tr.release();
  });
}

rss_status rss_tree_query(const rss_tree *tree, int what, void *buf, size_t *nbytes) {
  return guard([&] {
    if (!tree || !nbytes) throw Fail{RSS_EINVAL, "rss_tree_query: NULL argument"};
    const HTree &T = tree->t;
    std::vector<unsigned char> tmp;
    auto put = [&](const void *p, size_t nb) {
      tmp.resize(nb);
      if (nb) memcpy(tmp.data(), p, nb);
    };
    size_t nn = T.depth.size();
    if (what == 0) put(T.perm.data(), T.perm.size() * 8);
    else if (what == 1) put(T.depth.data(), nn * 4);
    else if (what == 2) put(T.parent.data(), nn * 4);
    else if (what == 3) put(T.coord.data(), nn * 12);
    else if (what == 4) put(T.start.data(), nn * 8);
    else if (what == 5) put(T.count.data(), nn * 8);
    else if (what == 6) {
      int64_t s[4] = {(int64_t)nn, T.maxdepth, T.n, T.dim};
      put(s, sizeof(s));
    } else if (what >= 100 && what < 100 + 21) {
      int t = what - 100;
      if (t > T.maxdepth) put(nullptr, 0);
      else put(T.level[t].data(), T.level[t].size() * 4);
    } else if (what >= 200 && what < 200 + 21) {
      int t = what - 200;
      std::vector<int> rec;
      if (t <= T.maxdepth) {
        // cells of depth t holding points
        std::vector<uint64_t> keys;
        const int dim = T.dim;
        for (int64_t g = 0; g < T.n; g++) {
          int64_t c[3] = {0, 0, 0};
          for (int d = 0; d < dim; d++) c[d] = cell_at(T.x[g * dim + d], t);
          keys.push_back(morton_key(c, dim, std::max(t, 1)));
        }
        std::sort(keys.begin(), keys.end());
        keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
        int64_t side = (int64_t)1 << t;
        for (int node : T.level[t]) {
          std::vector<int> nr, rg;
          int lim = dim == 3 ? 2 : 0;
          for (int dz = -lim; dz <= lim; dz++)
            for (int dy = -2; dy <= 2; dy++)
              for (int dx = -2; dx <= 2; dx++) {
                int m = std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz)));
                if (m == 0) continue;
                int64_t p[3] = {T.coord[3 * node] + dx, T.coord[3 * node + 1] + dy, T.coord[3 * node + 2] + dz};
                bool ok = true;
                for (int d = 0; d < dim; d++) ok = ok && p[d] >= 0 && p[d] < side;
                if (!ok || find_key(keys, morton_key(p, dim, std::max(t, 1))) < 0) continue;
                (m == 1 ? nr : rg).push_back(code5(dx, dy, dz, dim));
              }
          std::sort(nr.begin(), nr.end());
          std::sort(rg.begin(), rg.end());
          rec.push_back((int)nr.size());
          rec.push_back((int)rg.size());
          rec.insert(rec.end(), nr.begin(), nr.end());
          rec.insert(rec.end(), rg.begin(), rg.end());
        }
      }
      put(rec.data(), rec.size() * 4);
    } else {
      throw Fail{RSS_EINVAL, "rss_tree_query: unknown item"};
    }
    size_t cap = *nbytes;
    *nbytes = tmp.size();
    if (buf) {
      if (cap < tmp.size()) throw Fail{RSS_EINVAL, "rss_tree_query: buffer too small"};
      if (!tmp.empty()) memcpy(buf, tmp.data(), tmp.size());
    }
  });
}

rss_status rss_factor(const double *pts, int64_t n, int dim, rss_kernel kernel, double eps, int leaf_size,
                      const rss_options *opts, rss_factorization **out) {
  return guard([&] {
    if (!out || n < 0 || (dim != 2 && dim != 3) || leaf_size < 1 || (n > 0 && !pts) || !(eps >= 0.0) ||
        (kernel.kind != RSS_LAPLACE2D_LOG && kernel.kind != RSS_LAPLACE3D_INV))
      throw Fail{RSS_EINVAL, "rss_factor: bad arguments"};
    rss_options o{};
    if (opts) o = *opts;
    if (o.prec != RSS_FP64 && o.prec != RSS_MIXED) throw Fail{RSS_EINVAL, "rss_factor: bad precision"};
    cudaStream_t st = (cudaStream_t)o.stream;
    std::vector<double> h;
    fetch_points(pts, n, dim, h, st);
    std::unique_ptr<rss_factorization> res(new rss_factorization());
    auto setup = [&](auto *F) {
      F->st = st;
      F->n = n;
      F->dim = dim;
      F->tree.dim = dim;
      F->tree.leaf = leaf_size;
      F->tree.n = n;
      build_tree(F->tree, h.data());
      F->K.kind = kernel.kind;
      F->K.diag = kernel.diag;
      F->K.w = kernel.weight > 0 ? kernel.weight : (n > 0 ? 1.0 / (double)n : 1.0);
      F->px.np = o.n_proxy > 0 ? o.n_proxy : (dim == 2 ? 64 : 512);
      F->px.radius = o.proxy_radius > 0 ? o.proxy_radius : 2.5;
      F->eps = eps;
      run_factor(*F);
    };
    if (o.prec == RSS_FP64) {
      auto *F = new Factor<double>();
      res->impl.reset(F);
      F->prec = RSS_FP64;
      setup(F);
    } else {
      auto *F = new Factor<float>();
      res->impl.reset(F);
      F->prec = RSS_MIXED;
      setup(F);
    }
    *out = res.release();
  });
}

rss_status rss_apply(const rss_factorization *f, const double *x, double *y, int nrhs) {
  return sweep_entry(f, x, y, nrhs, false);
}

rss_status rss_solve(const rss_factorization *f, const double *b, double *x, int nrhs) {
  return sweep_entry(f, b, x, nrhs, true);
}

rss_status rss_matvec(const rss_factorization *f, const double *x, double *y, int nrhs) {
  return guard([&] {
    if (!f || !f->impl || nrhs < 1) throw Fail{RSS_EINVAL, "rss_matvec: bad arguments"};
    auto run = [&](const auto &F) {
      if (F.n > 0 && (!x || !y)) throw Fail{RSS_EINVAL, "NULL vector"};
      launch_matvec(ptr<double>(F.d_x), F.dim, F.K, ptr<int64_t>(F.d_perm), x, y, F.n, nrhs,
                    F.st);
      check_launch("matvec");
      CK(cudaStreamSynchronize(F.st));
    };
    if (f->impl->prec == RSS_FP64) run(static_cast<const Factor<double> &>(*f->impl));
    else run(static_cast<const Factor<float> &>(*f->impl));
  });
}

rss_status rss_stats(const rss_factorization *f, int64_t *buf, size_t *nbytes) {
  return guard([&] {
    if (!f || !f->impl || !nbytes) throw Fail{RSS_EINVAL, "rss_stats: bad arguments"};
    std::vector<int64_t> s;
    auto fill = [&](const auto &F) {
      s = {(int64_t)F.h_boxes.size(), F.ntop, F.factor_bytes, F.tree.maxdepth, F.n, F.prec};
      for (const auto &b : F.h_boxes) {
        s.push_back(b.depth);
        s.push_back(b.b);
        s.push_back(b.k);
        s.push_back(b.nj);
      }
    };
    if (f->impl->prec == RSS_FP64) fill(static_cast<const Factor<double> &>(*f->impl));
    else fill(static_cast<const Factor<float> &>(*f->impl));
    size_t need = s.size() * sizeof(int64_t), cap = *nbytes;
    *nbytes = need;
    if (buf) {
      if (cap < need) throw Fail{RSS_EINVAL, "rss_stats: buffer too small"};
      memcpy(buf, s.data(), need);
    }
  });
}

void rss_free(void *handle) {
  if (!handle) return;
  // both handle types start with a distinct 32-bit tag
  uint32_t magic = *static_cast<const uint32_t *>(handle);
  if (magic == MAGIC_TREE) delete static_cast<rss_tree *>(handle);
  else if (magic == MAGIC_FACTOR) delete static_cast<rss_factorization *>(handle);
}

}  // extern "C"
