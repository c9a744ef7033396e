// api.cu -- host orchestration and the C ABI (include/rss.h).
//
// The factorization follows Algorithm 1 of the paper: levels (tree depths)
// from the finest to depth 2, boxes of a level in colour-major order.  All
// arithmetic runs in the kernels of kernels.cu; the host builds the index
// structures of each level (which cells hold active DOFs, their neighbour
// tables and pair-block offsets) once the ranks of the previous level are
// known, and launches one ID / elimination / Schur launch per colour phase.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <map>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <unordered_map>
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

// Library-private stream-ordered memory pools, per device and kind: kind 0
// for long-lived data, kind 1 for the large per-level transients (pair-block
// pools, phase scratch) so that their blocks are reused whole from one
// factorization to the next instead of being split by small allocations.
// Freed memory stays in the pool (release threshold: never).
static cudaMemPool_t lib_pool(int kind = 0) {
  static std::mutex m;
  static cudaMemPool_t pools[64][2] = {};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Fail{RSS_ECUDA, "device index out of range"};
  std::lock_guard<std::mutex> lk(m);
  cudaMemPool_t &pool = pools[dev][kind];
  if (!pool) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    CK(cudaMemPoolCreate(&pool, &props));
    uint64_t thr = UINT64_MAX;
    CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
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
  void alloc(size_t nb, cudaStream_t s, int kind = 0) {
    release();
    st = s;
    bytes = nb;
    if (nb == 0) nb = 16;
    CK(cudaMallocFromPoolAsync(&p, nb, lib_pool(kind), s));
  }
  void release() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    bytes = 0;
  }
  // take over o's memory (o is left empty)
  void take(DBuf &o) {
    release();
    p = o.p;
    bytes = o.bytes;
    st = o.st;
    o.p = nullptr;
    o.bytes = 0;
  }
};

template <typename U> static inline U *ptr(const DBuf &b) { return static_cast<U *>(b.p); }

// Make d hold at least `bytes` (contents are not kept).
static void grow(DBuf &d, size_t bytes, cudaStream_t st, int kind = 0) {
  if (!d.p || d.bytes < bytes) d.alloc(bytes, st, kind);
}

// Host-to-device copies go through a per-thread pinned staging ring, so they
// are asynchronous DMA copies instead of pageable ones.  A region is reused
// only after the copies that read it have completed (an event per copy).
struct Staging {
  char *buf = nullptr;
  size_t cap = 0, off = 0;
  std::vector<cudaEvent_t> inflight, spare;
  void wait_all() {
    for (cudaEvent_t e : inflight) {
      cudaEventSynchronize(e);
      spare.push_back(e);
    }
    inflight.clear();
    off = 0;
  }
};
static thread_local Staging g_stage;

static void staged_h2d(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return;
  Staging &S = g_stage;
  const size_t need = (bytes + 255) & ~size_t(255);
  if (need > S.cap) {
    S.wait_all();
    if (S.buf) cudaFreeHost(S.buf);
    S.buf = nullptr;
    S.cap = 0;
    size_t cap = std::max<size_t>((size_t)16 << 20, 2 * need);
    CK(cudaHostAlloc((void **)&S.buf, cap, cudaHostAllocDefault));
    S.cap = cap;
  }
  if (S.off + need > S.cap) S.wait_all();
  memcpy(S.buf + S.off, src, bytes);
  CK(cudaMemcpyAsync(dst, S.buf + S.off, bytes, cudaMemcpyHostToDevice, st));
  cudaEvent_t e;
  if (S.spare.empty()) {
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  } else {
    e = S.spare.back();
    S.spare.pop_back();
  }
  CK(cudaEventRecord(e, st));
  S.inflight.push_back(e);
  S.off += need;
}

// Small arrays go through the staging ring; large ones are copied from the
// pageable vector directly (the copy has left the vector when the call
// returns, and on this platform it runs near memory speed, faster than a
// host copy into the ring first).
template <typename U> static void upload(DBuf &d, const std::vector<U> &h, cudaStream_t st) {
  const size_t nb = h.size() * sizeof(U);
  d.alloc(nb, st);
  if (nb == 0) return;
  if (nb <= ((size_t)256 << 10)) staged_h2d(d.p, h.data(), nb, st);
  else CK(cudaMemcpyAsync(d.p, h.data(), nb, cudaMemcpyHostToDevice, st));
}

// ---------------------------------------------------------------------------
// Host worker pool: parallel_for(n, f) runs f(0..n-1) on up to 16 threads
// created once per process (the calling thread works too).  Calls from
// several host threads are serialised; an exception in f is rethrown in the
// caller.
// ---------------------------------------------------------------------------

class HostPool {
 public:
  static HostPool &get() {
    static HostPool *p = new HostPool();  // never destroyed: workers end with the process
    return *p;
  }
  int size() const { return (int)th_.size() + 1; }
  void parallel_for(int64_t n, const std::function<void(int64_t)> &f) {
    if (n <= 0) return;
    if (n == 1 || th_.empty() || in_job()) {  // nested calls run inline
      for (int64_t i = 0; i < n; i++) f(i);
      return;
    }
    std::lock_guard<std::mutex> call(call_m_);
    {
      std::lock_guard<std::mutex> lk(m_);
      job_ = &f;
      njob_ = n;
      next_.store(0);
      err_ = nullptr;
      active_ = (int)th_.size();
      gen_++;
    }
    cv_.notify_all();
    run();
    std::unique_lock<std::mutex> lk(m_);
    done_cv_.wait(lk, [&] { return active_ == 0; });
    job_ = nullptr;
    if (err_) std::rethrow_exception(err_);
  }

 private:
  HostPool() {
    unsigned hw = std::thread::hardware_concurrency();
    int nt = (int)std::min<unsigned>(hw ? hw : 1, 16) - 1;
    for (int i = 0; i < nt; i++) {
      th_.emplace_back([this] { worker(); });
      th_.back().detach();
    }
  }
  static bool &in_job() {
    static thread_local bool f = false;
    return f;
  }
  void run() {
    in_job() = true;
    for (;;) {
      const int64_t i = next_.fetch_add(1);
      if (i >= njob_) break;
      try {
        (*job_)(i);
      } catch (...) {
        std::lock_guard<std::mutex> lk(m_);
        if (!err_) err_ = std::current_exception();
      }
    }
    in_job() = false;
  }
  void worker() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
      }
      run();
      std::lock_guard<std::mutex> lk(m_);
      if (--active_ == 0) done_cv_.notify_all();
    }
  }
  std::vector<std::thread> th_;
  std::mutex m_, call_m_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int64_t)> *job_ = nullptr;
  int64_t njob_ = 0;
  std::atomic<int64_t> next_{0};
  int active_ = 0;
  uint64_t gen_ = 0;
  std::exception_ptr err_;
};

// parallel_for over [0, n) in chunks of at least `grain` indices
template <typename F> static void parallel_range(int64_t n, int64_t grain, F &&f) {
  HostPool &P = HostPool::get();
  const int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>((n + grain - 1) / std::max<int64_t>(grain, 1),
                                                                4 * (int64_t)P.size()));
  if (nchunk <= 1) {
    f(0, n);
    return;
  }
  P.parallel_for(nchunk, [&](int64_t c) { f(n * c / nchunk, n * (c + 1) / nchunk); });
}

// ---------------------------------------------------------------------------
// Tree
// ---------------------------------------------------------------------------

static const uint32_t MAGIC_TREE = 0x52535354u, MAGIC_FACTOR = 0x52535346u, MAGIC_MLP = 0x5253534Du;

// Device state of the rank-proposal network: FP32 master parameters, their
// bfloat16 copy, Adam moments and step, gradient and loss.
struct MlpModel {
  cudaStream_t st = nullptr;
  DBuf theta, wbf, m, v, grad, step, loss;
};

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

// Bit spreading by shift-and-mask (same interleaving as morton_key, x in
// the lowest bit of each group), for up to 21 bits per coordinate.
static inline uint64_t spread2(uint64_t x) {
  x &= 0x1fffffULL;
  x = (x | (x << 16)) & 0x0000ffff0000ffffULL;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffULL;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0fULL;
  x = (x | (x << 2)) & 0x3333333333333333ULL;
  x = (x | (x << 1)) & 0x5555555555555555ULL;
  return x;
}
static inline uint64_t spread3(uint64_t x) {
  x &= 0x1fffffULL;
  x = (x | (x << 32)) & 0x001f00000000ffffULL;
  x = (x | (x << 16)) & 0x001f0000ff0000ffULL;
  x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
  x = (x | (x << 2)) & 0x1249249249249249ULL;
  return x;
}
static inline uint64_t morton_fast(const int64_t *c, int dim) {
  return dim == 2 ? (spread2(c[0]) | (spread2(c[1]) << 1))
                  : (spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2));
}
// The inverse: every dim-th bit of x from bit 0, packed.
static inline uint64_t compact2(uint64_t x) {
  x &= 0x5555555555555555ULL;
  x = (x | (x >> 1)) & 0x3333333333333333ULL;
  x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0fULL;
  x = (x | (x >> 4)) & 0x00ff00ff00ff00ffULL;
  x = (x | (x >> 8)) & 0x0000ffff0000ffffULL;
  x = (x | (x >> 16)) & 0x00000000ffffffffULL;
  return x;
}
static inline uint64_t compact3(uint64_t x) {
  x &= 0x1249249249249249ULL;
  x = (x | (x >> 2)) & 0x10c30c30c30c30c3ULL;
  x = (x | (x >> 4)) & 0x100f00f00f00f00fULL;
  x = (x | (x >> 8)) & 0x001f0000ff0000ffULL;
  x = (x | (x >> 16)) & 0x001f00000000ffffULL;
  x = (x | (x >> 32)) & 0x00000000001fffffULL;
  return x;
}
// Cell coordinates of a Morton key (x in the lowest bit of each group).
static inline void morton_cell(uint64_t k, int dim, int *c) {
  if (dim == 2) {
    c[0] = (int)compact2(k);
    c[1] = (int)compact2(k >> 1);
    c[2] = 0;
  } else {
    c[0] = (int)compact3(k);
    c[1] = (int)compact3(k >> 1);
    c[2] = (int)compact3(k >> 2);
  }
}

struct HTree {
  uint32_t magic = MAGIC_TREE;
  int dim = 2, leaf = 64, maxdepth = 0;
  int64_t n = 0;
  std::vector<int64_t> perm;
  std::vector<double> x;    // tree order
  std::vector<uint64_t> key;  // depth-20 Morton key of each DOF, tree order
  std::vector<int> c20;       // depth-20 integer cell of each DOF (dim per DOF), tree order
  std::vector<int> depth, parent, coord;
  std::vector<int64_t> start, count;
  std::vector<std::vector<int>> level;  // boxes per depth, elimination order
};

// Colour of a cell: sum_d (c_d mod base) base^d.  Base 3 (the default) puts
// same-colour cells >= 3 apart; base 2 is the paper's schedule (Sec. 5),
// same-colour cells >= 2 apart.
static int colour_of(const int *c, int dim, int base = 3) {
  int col = 0, mul = 1;
  for (int d = 0; d < dim; d++) {
    col += (c[d] % base) * mul;
    mul *= base;
  }
  return col;
}

// Elimination order of every depth: colour-major with 3^d colours, Morton
// order within a colour (nodes of a depth come in Morton order already).
static void level_lists(HTree &T) {
  const int dim = T.dim;
  T.level.assign(T.maxdepth + 1, {});
  for (int i = 0; i < (int)T.depth.size(); i++) T.level[T.depth[i]].push_back(i);
  std::vector<int> col(T.depth.size());
  for (size_t i = 0; i < T.depth.size(); i++) col[i] = colour_of(&T.coord[3 * i], dim);
  for (auto &lv : T.level) std::stable_sort(lv.begin(), lv.end(), [&](int a, int b) { return col[a] < col[b]; });
}

// Tree-order points of a single problem kept on the device by a factor:
// coordinates, the permutation (tree -> caller order) and depth-20 cells.
struct DevTreePoints {
  DBuf x, perm, c20, key;
  bool have = false;
};

// Trees of nprob problems (device points pts[p], n[p] each) built on the GPU
// (tree.cu) and copied to the host: one build over all problems when the
// problem index fits above the Morton key, else one build per group.  With
// `keep` (a single problem), the tree-order coordinates, permutation and
// cells stay on the device in *keep and are not copied to the host.
static void build_trees_gpu(std::vector<HTree> &trees, const double *const *pts, const int64_t *n, int nprob, int dim,
                            int leaf, cudaStream_t st, DevTreePoints *keep = nullptr) {
  if (nprob != 1) keep = nullptr;
  // problems per build: dim * 20 key bits plus the problem index within 64
  const int max_bits = 64 - dim * 20;
  const int per_build = max_bits >= 24 ? (1 << 24) : (1 << max_bits);
  for (int p0 = 0; p0 < nprob; p0 += per_build) {
    const int np = std::min(per_build, nprob - p0);
    std::vector<int64_t> pofs(np + 1, 0);
    for (int p = 0; p < np; p++) pofs[p + 1] = pofs[p] + n[p0 + p];
    const int64_t N = pofs[np];
    int bits = 0;
    while ((1 << bits) < np) bits++;
    DBuf d_pts, d_pofs, scratch;
    const double *P = pts[p0];
    if (np > 1 && N > 0) {
      d_pts.alloc(sizeof(double) * (size_t)N * dim, st, 1);
      for (int p = 0; p < np; p++)
        if (n[p0 + p] > 0)
          CK(cudaMemcpyAsync(ptr<double>(d_pts) + pofs[p] * dim, pts[p0 + p], sizeof(double) * n[p0 + p] * dim,
                             cudaMemcpyDeviceToDevice, st));
      P = ptr<double>(d_pts);
    }
    upload(d_pofs, pofs, st);
    TreeGpu G;
    G.pts = P;
    G.n = N;
    G.dim = dim;
    G.leaf = leaf;
    G.pofs = ptr<int64_t>(d_pofs);
    G.nprob = np;
    G.prob_bits = bits;
    scratch.alloc((size_t)tree_gpu_scratch_bytes(N, dim), st, 1);
    tree_gpu_sort(G, scratch.p, st);
    uint32_t nnode = 0;
    CK(cudaMemcpyAsync(&nnode, G.total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    DBuf o_depth, o_parent, o_coord, o_start, o_count, o_perm, o_x, o_c20, o_key;
    o_depth.alloc(sizeof(int) * std::max<uint32_t>(nnode, 1), st, 1);
    o_parent.alloc(sizeof(int) * std::max<uint32_t>(nnode, 1), st, 1);
    o_coord.alloc(sizeof(int) * 3 * std::max<uint32_t>(nnode, 1), st, 1);
    o_start.alloc(sizeof(int64_t) * std::max<uint32_t>(nnode, 1), st, 1);
    o_count.alloc(sizeof(int64_t) * std::max<uint32_t>(nnode, 1), st, 1);
    o_perm.alloc(sizeof(int64_t) * std::max<int64_t>(N, 1), st, 1);
    o_x.alloc(sizeof(double) * std::max<int64_t>(N, 1) * dim, st, 1);
    o_c20.alloc(sizeof(int) * std::max<int64_t>(N, 1) * dim, st, 1);
    o_key.alloc(sizeof(uint64_t) * std::max<int64_t>(N, 1), st, 1);
    tree_gpu_nodes(G, ptr<int>(o_depth), ptr<int>(o_parent), ptr<int>(o_coord), ptr<int64_t>(o_start),
                   ptr<int64_t>(o_count), ptr<int64_t>(o_perm), ptr<double>(o_x), ptr<int>(o_c20),
                   ptr<uint64_t>(o_key), st);
    check_launch("tree");
    std::vector<int> depth(nnode), parent(nnode), coord((size_t)3 * nnode);
    std::vector<int64_t> start(nnode), count(nnode), perm(keep ? 0 : N);
    std::vector<double> x(keep ? 0 : (size_t)N * dim);
    std::vector<int> c20(keep ? 0 : (size_t)N * dim);
    std::vector<uint64_t> key(N);
    auto d2h = [&](void *dst, const DBuf &src, size_t bytes) {
      if (bytes) CK(cudaMemcpyAsync(dst, src.p, bytes, cudaMemcpyDeviceToHost, st));
    };
    d2h(depth.data(), o_depth, sizeof(int) * nnode);
    d2h(parent.data(), o_parent, sizeof(int) * nnode);
    d2h(coord.data(), o_coord, sizeof(int) * 3 * nnode);
    d2h(start.data(), o_start, sizeof(int64_t) * nnode);
    d2h(count.data(), o_count, sizeof(int64_t) * nnode);
    if (keep) {
      keep->x.take(o_x);
      keep->perm.take(o_perm);
      keep->c20.take(o_c20);
      keep->have = true;
    } else {
      d2h(perm.data(), o_perm, sizeof(int64_t) * N);
      d2h(x.data(), o_x, sizeof(double) * N * dim);
      d2h(c20.data(), o_c20, sizeof(int) * N * dim);
    }
    d2h(key.data(), o_key, sizeof(uint64_t) * N);
    if (keep) keep->key.take(o_key);  // the copy above reads it first (stream order)
    CK(cudaStreamSynchronize(st));
    // split into the problems: a problem's nodes are contiguous (its points
    // are, and nodes are ordered by first point)
    int node0 = 0;
    for (int p = 0; p < np; p++) {
      HTree &T = trees[p0 + p];
      T.dim = dim;
      T.leaf = leaf;
      T.n = n[p0 + p];
      const int64_t off = pofs[p];
      int node1 = node0;
      while (node1 < (int)nnode && start[node1] < pofs[p + 1]) node1++;
      if (T.n == 0) node1 = node0;
      const int nn = node1 - node0;
      T.depth.assign(depth.begin() + node0, depth.begin() + node1);
      T.parent.resize(nn);
      T.start.resize(nn);
      T.count.assign(count.begin() + node0, count.begin() + node1);
      T.coord.assign(coord.begin() + 3 * (size_t)node0, coord.begin() + 3 * (size_t)node1);
      T.maxdepth = 0;
      for (int i = 0; i < nn; i++) {
        T.parent[i] = parent[node0 + i] < 0 ? -1 : parent[node0 + i] - node0;
        T.start[i] = start[node0 + i] - off;
        T.maxdepth = std::max(T.maxdepth, T.depth[i]);
      }
      if (nn == 0) {
        // an empty problem: a root of depth 0 holding nothing
        T.depth = {0};
        T.parent = {-1};
        T.coord = {0, 0, 0};
        T.start = {0};
        T.count = {0};
      }
      if (np == 1) {  // the whole build is this problem's
        T.perm.swap(perm);
        T.x.swap(x);
        T.c20.swap(c20);
        T.key.swap(key);
      } else {
        T.perm.resize(T.n);
        for (int64_t g = 0; g < T.n; g++) T.perm[g] = perm[off + g] - off;
        T.x.assign(x.begin() + off * dim, x.begin() + (off + T.n) * dim);
        T.c20.assign(c20.begin() + off * dim, c20.begin() + (off + T.n) * dim);
        T.key.assign(key.begin() + off, key.begin() + off + T.n);
      }
      level_lists(T);
      node0 = node1;
    }
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
  // a level built on the device: the cell tables stay there; per box its b,
  // |J|, ID rows inside the proxy surface and near / ring cells present
  bool on_device = false;
  int64_t ndof = 0;
  std::vector<int> box_b, box_nj, box_ring, box_nnc, box_nrc;
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

static HLevel build_level(const HTree &T, int t, const std::vector<int64_t> &active, int cbase = 3) {
  HLevel L;
  L.t = t;
  L.dim = T.dim;
  const int dim = T.dim;
  L.NB = dim == 2 ? 25 : 125;
  const size_t na = active.size();
  // depth-t key of a DOF from its depth-20 one: the Morton key drops dim
  // bits per level, and its coordinates are floor(v 2^20) >> (20 - t) =
  // floor(v 2^t), the DOF's depth-t cell (clamping included)
  const int ksh = dim * (20 - t);
  std::vector<uint64_t> dk(na);
  std::atomic<bool> unsorted{false};
  parallel_range((int64_t)na, (int64_t)1 << 15, [&](int64_t lo, int64_t hi) {
    for (int64_t q = lo; q < hi; q++) dk[q] = T.key[active[q]] >> ksh;
    for (int64_t q = std::max<int64_t>(lo, 1); q < hi; q++)
      if (dk[q] < dk[q - 1]) unsorted = true;
  });
  for (int64_t q0 = 1; q0 < (int64_t)na; q0++)  // chunk boundaries and anything missed
    if (dk[q0] < dk[q0 - 1]) {
      unsorted = true;
      break;
    }
  const bool sorted = !unsorted;
  std::vector<int> cid;
  if (sorted && na >= ((size_t)1 << 16)) {
    // cells are runs of the (tree-ordered) active list: cell c holds
    // active[start_c .. start_{c+1}) in order
    // run starts, found per chunk and concatenated in chunk order
    const int64_t nch = std::min<int64_t>(64, ((int64_t)na + (1 << 14) - 1) >> 14);
    std::vector<std::vector<int64_t>> part(nch);
    HostPool::get().parallel_for(nch, [&](int64_t h) {
      const int64_t lo = (int64_t)na * h / nch, hi = (int64_t)na * (h + 1) / nch;
      for (int64_t q = lo; q < hi; q++)
        if (q == 0 || dk[q] != dk[q - 1]) part[h].push_back(q);
    });
    std::vector<int64_t> starts;
    size_t ns = 0;
    for (const auto &v : part) ns += v.size();
    starts.reserve(ns);
    for (const auto &v : part) starts.insert(starts.end(), v.begin(), v.end());
    L.ncell = (int)starts.size();
    L.key.resize(L.ncell);
    L.cell_b.resize(L.ncell);
    L.cell_dof_off.resize(L.ncell + 1);
    L.cell_coord.assign(3 * (size_t)L.ncell, 0);
    L.cell_dofs.assign(active.begin(), active.end());
    L.cell_dof_off[L.ncell] = (int64_t)na;
    parallel_range(L.ncell, 4096, [&](int64_t c0, int64_t c1) {
      for (int64_t c = c0; c < c1; c++) {
        const int64_t q = starts[c], e = c + 1 < L.ncell ? starts[c + 1] : (int64_t)na;
        L.key[c] = dk[q];
        L.cell_b[c] = (int)(e - q);
        L.cell_dof_off[c] = q;
        morton_cell(dk[q], dim, &L.cell_coord[3 * c]);
      }
    });
  } else if (sorted) {
    cid.resize(na);
    // cells are runs of the (tree-ordered) active list: no sort needed
    for (size_t q = 0; q < na; q++) {
      if (q == 0 || dk[q] != dk[q - 1]) L.key.push_back(dk[q]);
      cid[q] = (int)L.key.size() - 1;
    }
  } else {
    cid.resize(na);
    L.key = dk;
    std::sort(L.key.begin(), L.key.end());
    L.key.erase(std::unique(L.key.begin(), L.key.end()), L.key.end());
    for (size_t q = 0; q < na; q++) cid[q] = find_key(L.key, dk[q]);
  }
  if (!cid.empty()) {
    L.ncell = (int)L.key.size();
    L.cell_b.assign(L.ncell, 0);
    for (size_t q = 0; q < na; q++) L.cell_b[cid[q]]++;
    L.cell_dof_off.assign(L.ncell + 1, 0);
    for (int c = 0; c < L.ncell; c++) L.cell_dof_off[c + 1] = L.cell_dof_off[c] + L.cell_b[c];
    L.cell_dofs.resize(na);
    L.cell_coord.assign(3 * L.ncell, 0);
    std::vector<int64_t> fill(L.cell_dof_off.begin(), L.cell_dof_off.end() - 1);
    for (size_t q = 0; q < na; q++) {
      int c = cid[q];
      if (fill[c] == L.cell_dof_off[c]) morton_cell(dk[q], dim, &L.cell_coord[3 * c]);
      L.cell_dofs[fill[c]++] = active[q];
    }
  } else if (na == 0) {
    L.ncell = 0;
    L.cell_dof_off.assign(1, 0);
  }
  L.cell_nbr.assign((size_t)L.ncell * L.NB, -1);
  L.pair_off.assign((size_t)L.ncell * L.NB, -1);
  const int64_t side = (int64_t)1 << t;
  // dense cell lookup when the level grid is small enough, else binary search
  int64_t grid_cells = 1;
  for (int d = 0; d < dim; d++) grid_cells *= side;
  std::vector<int> dense;
  if (grid_cells <= ((int64_t)1 << 24)) {
    dense.assign(grid_cells, -1);
    parallel_range(L.ncell, 8192, [&](int64_t c0, int64_t c1) {
      for (int64_t c = c0; c < c1; c++) {
        int64_t lin = 0, mul = 1;
        for (int d = 0; d < dim; d++) lin += (int64_t)L.cell_coord[3 * c + d] * mul, mul *= side;
        dense[lin] = (int)c;  // distinct cells, distinct entries
      }
    });
  }
  auto lookup = [&](const int64_t *p) -> int {
    if (!dense.empty()) {
      int64_t lin = 0, mul = 1;
      for (int d = 0; d < dim; d++) lin += p[d] * mul, mul *= side;
      return dense[lin];
    }
    return find_key(L.key, morton_fast(p, dim));
  };
  // neighbours at Chebyshev distance <= 2, then the pair-block offsets: a
  // cell's blocks in code order, cells in order
  std::vector<int64_t> psum(L.ncell + 1, 0);
  parallel_range(L.ncell, 2048, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; c++) {
      int64_t tot = 0;
      int lim = dim == 3 ? 2 : 0;
      for (int dz = -lim; dz <= lim; dz++)
        for (int dy = -2; dy <= 2; dy++)
          for (int dx = -2; dx <= 2; dx++) {
            int64_t p[3] = {L.cell_coord[3 * c] + dx, L.cell_coord[3 * c + 1] + dy, L.cell_coord[3 * c + 2] + dz};
            bool ok = true;
            for (int d = 0; d < dim; d++) ok = ok && p[d] >= 0 && p[d] < side;
            if (!ok) continue;
            int nb = lookup(p);
            if (nb < 0) continue;
            L.cell_nbr[(size_t)c * L.NB + code5(dx, dy, dz, dim)] = nb;
            tot += (int64_t)L.cell_b[c] * L.cell_b[nb];
          }
      psum[c + 1] = tot;
    }
  });
  for (int c = 0; c < L.ncell; c++) {
    psum[c + 1] += psum[c];
    L.bmax = std::max(L.bmax, L.cell_b[c]);
  }
  parallel_range(L.ncell, 2048, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; c++) {
      int64_t off = psum[c];
      for (int code = 0; code < L.NB; code++) {
        const int nb = L.cell_nbr[(size_t)c * L.NB + code];
        if (nb < 0) continue;
        L.pair_off[(size_t)c * L.NB + code] = off;
        off += (int64_t)L.cell_b[c] * L.cell_b[nb];
      }
    }
  });
  L.pool_elems = psum[L.ncell];
  for (int node : T.level[t]) {
    int64_t p[3] = {T.coord[3 * node], T.coord[3 * node + 1], T.coord[3 * node + 2]};
    int c = find_key(L.key, morton_fast(p, dim));
    if (c < 0) continue;  // every DOF of the box has become inactive
    L.box_cell.push_back(c);
    L.box_node.push_back(node);
    L.box_colour.push_back(colour_of(&T.coord[3 * node], dim, cbase));
  }
  if (cbase != 3) {
    // colour-major with cbase^dim colours, Morton order within a colour:
    // nodes of one depth in pre-order are in Morton order, so the boxes
    // sorted by node index, then a stable counting sort by colour
    const int nb = (int)L.box_cell.size();
    std::vector<int> byn(nb), ord(nb);
    for (int q = 0; q < nb; q++) byn[q] = q;
    std::sort(byn.begin(), byn.end(), [&](int a, int b) { return L.box_node[a] < L.box_node[b]; });
    int ncol = 1;
    for (int d = 0; d < dim; d++) ncol *= cbase;
    std::vector<int> cstart(ncol + 1, 0);
    for (int q = 0; q < nb; q++) cstart[L.box_colour[q] + 1]++;
    for (int c = 0; c < ncol; c++) cstart[c + 1] += cstart[c];
    for (int q : byn) ord[cstart[L.box_colour[q]]++] = q;
    std::vector<int> bc(nb), bn(nb), bcol(nb);
    for (int q = 0; q < nb; q++) bc[q] = L.box_cell[ord[q]], bn[q] = L.box_node[ord[q]], bcol[q] = L.box_colour[ord[q]];
    L.box_cell.swap(bc);
    L.box_node.swap(bn);
    L.box_colour.swap(bcol);
  }
  return L;
}

// ---------------------------------------------------------------------------
// Factor
// ---------------------------------------------------------------------------

struct Phase {
  int first, count, bmax, njmax;
  int wfirst = 0, wcount = 0;  // solve-sweep work items (box, chunk of J)
  int shared = 0;              // 1: boxes of the phase may share near DOFs (2^d colours)
};

// Per-kernel-class timing with CUDA events on the launching stream, plus the
// algorithmic bytes and flops of each launch (filled in once the ranks of the
// boxes it handled are known).
enum KClass {
  KC_ASSEMBLE, KC_ID, KC_ELIM, KC_SCHUR, KC_TOPLU, KC_SWEEP, KC_TOP, KC_PERMUTE,
  KC_HOST_TREE, KC_HOST_LEVEL, KC_HOST_WAIT, KC_REFINE_OP, KC_INNER_OP, KC_N
};

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
  int first, count, nrhs;
  double bytes, flops;
};

struct Prof {
  bool on = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> spare;
  double ms[KC_N] = {}, bytes[KC_N] = {}, flops[KC_N] = {};
  int64_t launches[KC_N] = {};
  cudaEvent_t ev() {
    if (!spare.empty()) {
      cudaEvent_t e = spare.back();
      spare.pop_back();
      return e;
    }
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    return e;
  }
  int begin(int cls, cudaStream_t st, int first = 0, int count = 0, int nrhs = 0, double bytes_ = 0,
            double flops_ = 0) {
    if (!on) return -1;
    ProfRec r{cls, ev(), ev(), first, count, nrhs, bytes_, flops_};
    CK(cudaEventRecord(r.a, st));
    pending.push_back(r);
    return (int)pending.size() - 1;
  }
  void end(int idx, cudaStream_t st) {
    if (idx >= 0) CK(cudaEventRecord(pending[idx].b, st));
  }
  void reset() {
    for (int c = 0; c < KC_N; c++) ms[c] = bytes[c] = flops[c] = 0, launches[c] = 0;
  }
  // host wall-clock intervals (tree build, level preparation, waits)
  void host(int cls, double msv) {
    if (!on) return;
    ms[cls] += msv;
    launches[cls] += 1;
  }
  ~Prof() {
    for (auto &r : pending) cudaEventDestroy(r.a), cudaEventDestroy(r.b);
    for (auto e : spare) cudaEventDestroy(e);
  }
};

struct FactorBase {
  uint32_t magic = MAGIC_FACTOR;
  int prec = 0;
  mutable Prof prof;
  virtual ~FactorBase() {}
};

template <typename T> struct Factor : FactorBase {
  using value_type = T;
  // one or more independent problems, DOFs concatenated in problem order
  std::vector<HTree> trees;
  std::vector<int64_t> pdof;  // DOF offset of each problem (nprob + 1)
  std::vector<double> pw;     // weight w of each problem
  int nprob = 1, maxdepth = 0;
  KernelParams K{};
  ProxyParams px{};
  double eps = 0;
  int flags = 0;
  cudaStream_t st = nullptr;
  int64_t n = 0;
  int dim = 2;
  DBuf d_x, d_perm, d_cell, d_off, d_err, d_proxy, d_wdof;  // d_proxy: unit proxy points in T
  DevTreePoints dev_pts;  // a single problem's tree-order points, kept on the device
  Points P{};
  std::vector<std::unique_ptr<DBuf>> store;  // factor storage chunks
  int64_t factor_bytes = 0;
  DBuf d_boxes;
  std::vector<FBox<T>> h_boxes;
  std::vector<Phase> phases;
  // top blocks, one per problem
  int ntop = 0;  // total over problems
  std::vector<int> h_tn;
  std::vector<int64_t> h_toff, h_loff;
  DBuf d_top, d_topLU, d_toppiv, d_tn, d_toff, d_loff;
  DBuf d_topinv;  // one problem's U^{-1} L^{-1} of the top block (ntop <= 1024), else empty
  mutable DBuf d_work, d_topwork;
  // Cholesky factors of the diagonal blocks for the generalized square root
  // (rss_sqrt_apply), built on its first use
  mutable DBuf d_chol, d_coff, d_cerr;
  mutable bool chol_ready = false;
  mutable int chol_rmax = 0;
  mutable int work_nrhs = 0, work_gen = 0;
  // solve sweeps captured in a CUDA graph, one per nrhs <= 4, replayed with
  // fixed input/output buffers (options.use_graphs)
  bool use_graphs = false;
  struct SweepGraph {
    int gen = -1, kernels = 0;
    cudaGraphExec_t exec = nullptr;
  };
  mutable SweepGraph sgraph[5];
  mutable DBuf g_in, g_out;
  // asynchronous factors (RSS_FLAG_ASYNC): the device error flag as copied
  // behind the last call's work, and the event that marks the copy done
  mutable int *h_err = nullptr;
  mutable cudaEvent_t ev_err = nullptr;
  mutable bool err_pending = false;
  bool async() const { return (flags & RSS_FLAG_ASYNC) != 0 && !prof.on; }
  ~Factor() {
    for (auto &g : sgraph)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    if (ev_err) cudaEventDestroy(ev_err);
    if (h_err) cudaFreeHost(h_err);
  }
  // FP64 residual operator: FFT convolution when a single problem's points
  // are the cell centres of a regular grid, direct summation otherwise
  int grid_side = 0;
  std::vector<int64_t> grid_index;  // caller order
  mutable GridOp G;
  mutable DBuf g_gidx, g_C, g_X, g_tw;
  mutable DBuf g_Cf, g_Xf, g_twf;  // FP32 copies for the inner GMRES products
  mutable bool grid_ready = false, grid_f32_ready = false;
  int mv_ntile = 0;
  DBuf d_mv_ts, d_mv_te, d_mv_sb, d_mv_se;
  // rank proposal: the network (borrowed during rss_factor only), the
  // features of every box (MLP_NFEAT each, box order) and storage accounting
  // solve sweeps: work items (box, chunk) of every phase, per-box counters,
  // partial sums of the backward sweep
  DBuf d_wbox, d_wchunk, d_wcnt, d_pbuf, d_poff;
  const struct MlpModel *mlp = nullptr;
  std::vector<float> feats;
  int64_t reserved_T = 0, used_T = 0, ovf_used = 0;  // elements of T
  int retries = 0;
  DBuf d_ovf_used;

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
  F.work_gen++;  // captured sweeps hold the old buffers
}

// Algorithmic work of one launch over boxes [first, first+count):
//   ID     : Householder reduction of the m x b ID matrix (m = |O| + n_p):
//            2 m b^2 flops; bytes = the |O| x b rows read + T written.
//   ELIM   : X_JR, X_RJ (2 * 2 nj k r), X_RR (4 r^2 k), LU (2/3 r^3), E and G
//            solves (2 * 2 nj r^2) flops; bytes = A_BB + near rows/columns
//            read, E, G, LU written.
//   SCHUR  : 2 nj^2 r flops; bytes = nj^2 read + written, E and X_RJ read.
//   SWEEP  : 2 nrhs (k r + 2 nj r + r^2) flops; bytes = the factor's
//            T, E, G, LU read once + the vector entries touched.
template <typename T> static void prof_collect(const Factor<T> &F) {
  Prof &P = F.prof;
  if (P.pending.empty()) return;
  const double sz = sizeof(T);
  for (auto &r : P.pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    double bytes = r.bytes, flops = r.flops;
    const bool per_box = r.cls == KC_ID || r.cls == KC_ELIM || r.cls == KC_SCHUR || r.cls == KC_SWEEP;
    for (int q = r.first; per_box && q < r.first + r.count; q++) {
      const FBox<T> &b = F.h_boxes[q];
      double B = b.b, k = b.k, rr = b.r, nj = b.nj, no = b.no, m = b.no + F.px.np;
      if (r.cls == KC_ID) {
        flops += 2.0 * m * B * B;
        bytes += (no * B + k * rr) * sz + B * 8.0;
      } else if (r.cls == KC_ELIM) {
        flops += 4.0 * nj * k * rr + 4.0 * rr * rr * k + 2.0 / 3.0 * rr * rr * rr + 4.0 * nj * rr * rr;
        bytes += (B * B + 2.0 * (nj - k) * B + 2.0 * nj * rr + rr * rr) * sz;
      } else if (r.cls == KC_SCHUR) {
        flops += 2.0 * nj * nj * rr;
        bytes += (2.0 * nj * nj + 2.0 * nj * rr) * sz;
      } else if (r.cls == KC_SWEEP) {
        flops += 2.0 * r.nrhs * (k * rr + 2.0 * nj * rr + rr * rr);
        bytes += (k * rr + 2.0 * nj * rr + rr * rr) * sz + 2.0 * (nj + rr) * r.nrhs * sz;
      }
    }
    P.ms[r.cls] += ms;
    P.bytes[r.cls] += bytes;
    P.flops[r.cls] += flops;
    P.launches[r.cls] += 1;
    P.spare.push_back(r.a);
    P.spare.push_back(r.b);
  }
  P.pending.clear();
}

static inline double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int check_err(DBuf &d_err, cudaStream_t st) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return h;
}

// Asynchronous factors (RSS_FLAG_ASYNC).  A call that leaves device work
// whose error flag nobody has read queues a copy of the flag into pinned
// host memory behind that work, with an event (defer_err); the next call on
// the factor reads it once the event has completed, or rss_sync waits for
// it, and reports what the device recorded (take_deferred).
template <typename T> static void defer_err(const T &F) {
  if (!F.h_err) {
    CK(cudaHostAlloc((void **)&F.h_err, sizeof(int), cudaHostAllocDefault));
    *F.h_err = 0;
    CK(cudaEventCreateWithFlags(&F.ev_err, cudaEventDisableTiming));
  }
  CK(cudaMemcpyAsync(F.h_err, F.d_err.p, sizeof(int), cudaMemcpyDeviceToHost, F.st));
  CK(cudaEventRecord(F.ev_err, F.st));
  F.err_pending = true;
}
template <typename T> static void take_deferred(const T &F, bool wait) {
  if (!F.err_pending) return;
  if (wait) {
    CK(cudaEventSynchronize(F.ev_err));
  } else {
    const cudaError_t q = cudaEventQuery(F.ev_err);
    if (q == cudaErrorNotReady) return;  // still running: a later call reports it
    CK(q);
  }
  F.err_pending = false;
  const int e = *F.h_err;
  if (!e) return;
  *F.h_err = 0;
  CK(cudaMemsetAsync(F.d_err.p, 0, sizeof(int), F.st));
  if (e == DERR_NUMERIC) throw Fail{RSS_ENUMERIC, "zero pivot in the top block (reported after an asynchronous call)"};
  throw Fail{RSS_ECUDA, "device-side consistency check failed (reported after an asynchronous call)"};
}

// Points exactly at the cell centres ((i + 1/2) / s) of an s^dim grid, s a
// power of two, each cell used once: record every point's grid index.
template <typename T> static void detect_grid(Factor<T> &F) {
  F.grid_side = 0;
  if (F.nprob != 1) return;
  const HTree &T_ = F.trees[0];
  const int dim = T_.dim;
  const int64_t n = T_.n;
  F.grid_side = 0;
  if (n < 8) return;
  int64_t s = (int64_t)llround(pow((double)n, 1.0 / dim));
  int64_t tot = 1;
  for (int d = 0; d < dim; d++) tot *= s;
  if (tot != n || (s & (s - 1)) != 0 || 2 * s > 2048) return;
  if (T_.x.empty()) {  // the points are on the device only: test them there
    DBuf seen, bad;
    seen.alloc(sizeof(unsigned) * (size_t)n, F.st);
    bad.alloc(sizeof(int), F.st);
    F.g_gidx.alloc(sizeof(int64_t) * (size_t)n, F.st);
    CK(cudaMemsetAsync(seen.p, 0, sizeof(unsigned) * (size_t)n, F.st));
    CK(cudaMemsetAsync(bad.p, 0, sizeof(int), F.st));
    grid_detect(ptr<double>(F.d_x), ptr<int64_t>(F.d_perm), n, dim, s, ptr<int64_t>(F.g_gidx), ptr<unsigned>(seen),
                ptr<int>(bad), F.st);
    check_launch("grid detection");
    if (check_err(bad, F.st) == 0) F.grid_side = (int)s;
    return;
  }
  std::vector<int64_t> gi(n);
  std::vector<unsigned char> seen(n, 0);
  std::atomic<bool> bad{false};
  parallel_range(n, (int64_t)1 << 15, [&](int64_t lo, int64_t hi) {
    for (int64_t g = lo; g < hi && !bad.load(std::memory_order_relaxed); g++) {
      int64_t lin = 0, mul = 1;
      for (int d = 0; d < dim; d++) {
        double v = T_.x[g * dim + d] * (double)s - 0.5;
        double iv = nearbyint(v);
        if (v != iv || iv < 0 || iv >= (double)s) {
          bad = true;
          return;
        }
        lin += (int64_t)iv * mul;
        mul *= s;
      }
      if (__atomic_exchange_n(&seen[lin], (unsigned char)1, __ATOMIC_RELAXED)) {  // a cell used twice
        bad = true;
        return;
      }
      gi[T_.perm[g]] = lin;
    }
  });
  if (bad) return;
  F.grid_side = (int)s;
  F.grid_index.swap(gi);
}

// Merge the depth-t cells of several problems into one level: cell ids,
// DOF ids (problem offset), neighbour tables, pair-block offsets and boxes
// are shifted; cells of different problems are never neighbours.  Boxes are
// ordered colour-major over all problems (each problem keeps its own order
// within a colour).
static void append_level(HLevel &H, const HLevel &Hp, int64_t dof_off, std::vector<int> &box_prob, int prob) {
  const int cbase = H.ncell;
  const int64_t dbase = H.cell_dofs.size(), pbase = H.pool_elems;
  if (H.cell_dof_off.empty()) H.cell_dof_off.push_back(0);
  for (int c = 0; c < Hp.ncell; c++) {
    H.cell_b.push_back(Hp.cell_b[c]);
    H.cell_dof_off.push_back(dbase + Hp.cell_dof_off[c + 1]);
    for (int d = 0; d < 3; d++) H.cell_coord.push_back(Hp.cell_coord[3 * c + d]);
    for (int o = 0; o < Hp.NB; o++) {
      int nb = Hp.cell_nbr[(size_t)c * Hp.NB + o];
      H.cell_nbr.push_back(nb >= 0 ? nb + cbase : -1);
      int64_t po = Hp.pair_off[(size_t)c * Hp.NB + o];
      H.pair_off.push_back(po >= 0 ? po + pbase : -1);
    }
  }
  for (int64_t g : Hp.cell_dofs) H.cell_dofs.push_back(g + dof_off);
  for (size_t q = 0; q < Hp.box_cell.size(); q++) {
    H.box_cell.push_back(Hp.box_cell[q] + cbase);
    H.box_node.push_back(Hp.box_node[q]);
    H.box_colour.push_back(Hp.box_colour[q]);
    box_prob.push_back(prob);
  }
  H.ncell += Hp.ncell;
  H.pool_elems += Hp.pool_elems;
  H.bmax = std::max(H.bmax, Hp.bmax);
}

// ---------------------------------------------------------------------------
// Autotuner: the ID kernel's launch shape -- threads per column (each
// thread keeps 32 rows (FP32) of every panel, so more threads per column
// mean taller panels and fewer sequential reflector steps) and fold groups
// per box (how many thread groups split a box's rows) -- trades latency per
// box against boxes resident per SM; the best shape depends on the box width
// and the number of boxes in a colour phase.  The first phase that meets a (precision, width class,
// phase-size class) key times every candidate on that phase (the ID launch
// is idempotent: it only writes the boxes' ID results), keeps the fastest
// for the rest of the process and re-runs it, so every factorization with
// that key computes exactly the same thing.
// ---------------------------------------------------------------------------

// Candidate launch shapes (threads per column, fold groups per box, CTAs per
// box, panel rows per thread in units of 32 FP32 / 16 FP64 rows); threads
// per column 0 is the warp-per-panel kernel with `groups` warps per box
// (width class 64 only); two units of rows only with one thread per column.
constexpr int kNShapes = 18;
static const int kTuneShapes[kNShapes][4] = {
    {1, 1, 1, 1}, {1, 2, 1, 1}, {1, 4, 1, 1}, {2, 1, 1, 1}, {2, 2, 1, 1}, {2, 4, 1, 1},
    {4, 1, 1, 1}, {4, 2, 1, 1}, {2, 1, 4, 1}, {2, 1, 8, 1}, {4, 1, 4, 1}, {4, 1, 8, 1},
    {0, 2, 1, 1}, {0, 4, 1, 1}, {0, 8, 1, 1}, {1, 1, 1, 2}, {1, 2, 1, 2}, {1, 4, 1, 2}};
static bool shape_fits(int width, int tpc, int g, int rows = 1) {
  if (rows != 1 && (rows != 2 || tpc != 1 || width > 128)) return false;
  if (tpc == 0) return width == 64 && (g == 2 || g == 4 || g == 8);
  return width * tpc * g <= (tpc == 1 ? 256 : 512);
}
static int shape_hint(int c) {
  if (kTuneShapes[c][0] == 0) {  // warps as a power of two
    int lg = 0;
    while ((1 << lg) < kTuneShapes[c][1]) lg++;
    return (1 << 12) | lg;
  }
  return (kTuneShapes[c][3] == 2 ? 1 << 13 : 0) | (kTuneShapes[c][2] << 8) | (kTuneShapes[c][0] << 4) |
         kTuneShapes[c][1];
}
struct TuneEntry {
  int shape;            // index into kTuneShapes
  float us[kNShapes];   // time of each candidate, microseconds; 0 if not a candidate
};
static std::mutex g_tune_m;
static std::map<std::tuple<int, int, int>, TuneEntry> g_tune;

template <typename T, typename Launch>
static void tuned_id_launch(Factor<T> &F, int bmax, int nbox, Launch &&launch) {
  const bool tunable = bmax > 0 && bmax <= 256 && !(F.flags & RSS_FLAG_NO_AUTOTUNE);
  if (!tunable) {
    set_id_groups(0);
    launch();
    return;
  }
  int bucket = 0;
  while ((2 << bucket) <= nbox) bucket++;
  const int width = bmax <= 64 ? 64 : (bmax <= 128 ? 128 : 256);
  const auto key = std::make_tuple((int)sizeof(T), width, bucket);
  int shape = -1;
  {
    std::lock_guard<std::mutex> lk(g_tune_m);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) shape = it->second.shape;
  }
  if (shape < 0) {
    TuneEntry te{-1, {}};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 0.f;
    for (int ci = 0; ci < kNShapes; ci++) {
      const int tpc = kTuneShapes[ci][0], g = kTuneShapes[ci][1], ctas = kTuneShapes[ci][2];
      if (!shape_fits(width, tpc, g, kTuneShapes[ci][3])) continue;  // the kernels' thread limits
      if (ctas > 1 && width == 256 && tpc != 2) continue;  // the widest class: two threads per column
      set_id_groups(shape_hint(ci));
      float ms = 0.f;
      for (int rep = 0; rep < 2; rep++) {  // the second launch is timed
        CK(cudaEventRecord(e0, F.st));
        launch();
        CK(cudaEventRecord(e1, F.st));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
      }
      te.us[ci] = std::max(1e3f * ms, 1e-3f);
      if (te.shape < 0 || ms < best) {
        best = ms;
        te.shape = ci;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_tune_m);
    auto ins = g_tune.insert({key, te});
    shape = ins.first->second.shape;  // another thread may have tuned the key first
  }
  set_id_groups(shape_hint(shape));
  launch();
  set_id_groups(0);
}

// The elimination's launch shape (the k_elim2 path, boxes up to 128 wide):
// E and G formed in the same kernel (one CTA per box), or X_JR and X_RJ
// left in the scratch for the phase-wide k_elim_gemm with 1, 2, 4 or 8 CTAs
// per box sharing a box's rows of J.  Tuned like the ID, per (precision,
// width class, phase-size class): the elimination of a phase only writes
// its boxes' records, its scratch and its cells' active lists, the same
// values however often it runs, so re-running it on the first phase of a
// key is safe.  Not tuned with a rank proposal (its storage claims are
// counted) or on the forced large-box path.
constexpr int kNElim = 5;
static const int kElimShapes[kNElim][2] = {{0, 1}, {1, 1}, {1, 2}, {1, 4}, {1, 8}};  // (split, CTAs per box)
struct ElimTuneEntry {
  int shape;
  float us[kNElim];
};
static std::map<std::tuple<int, int, int>, ElimTuneEntry> g_tune_elim;  // guarded by g_tune_m

template <typename T, typename Launch>
static void tuned_elim_launch(Factor<T> &F, int bmax, int nbox, Launch &&launch) {
  const bool tunable = bmax > 0 && bmax <= 128 && !F.mlp && !(F.flags & RSS_FLAG_NO_AUTOTUNE);
  if (!tunable) {
    set_elim_shape(0);
    launch();
    return;
  }
  int bucket = 0;
  while ((2 << bucket) <= nbox) bucket++;
  const auto key = std::make_tuple((int)sizeof(T), bmax <= 64 ? 64 : 128, bucket);
  int shape = -1;
  {
    std::lock_guard<std::mutex> lk(g_tune_m);
    auto it = g_tune_elim.find(key);
    if (it != g_tune_elim.end()) shape = it->second.shape;
  }
  auto hint = [](int c) { return (kElimShapes[c][0] << 4) | kElimShapes[c][1]; };
  if (shape < 0) {
    ElimTuneEntry te{-1, {}};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 0.f;
    for (int ci = 0; ci < kNElim; ci++) {
      set_elim_shape(hint(ci));
      float ms = 0.f;
      for (int rep = 0; rep < 2; rep++) {  // the second launch is timed
        CK(cudaEventRecord(e0, F.st));
        launch();
        CK(cudaEventRecord(e1, F.st));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
      }
      te.us[ci] = std::max(1e3f * ms, 1e-3f);
      if (te.shape < 0 || ms < best) {
        best = ms;
        te.shape = ci;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_tune_m);
    auto ins = g_tune_elim.insert({key, te});
    shape = ins.first->second.shape;
  }
  set_elim_shape(hint(shape));
  launch();
  set_elim_shape(0);
}

// A level ran out of overflow space for boxes whose rank exceeded the
// proposed reservation: the factorization is redone with full reservations.
struct Retry {};

// Features of a box for the rank proposal, all known before its ID runs:
//   0 dim == 3            1 kernel kind          2 -log10(eps) / 10
//   3 log2(1 + b) / 10    4 log2(1 + |N|) / 10   5 log2(1 + |O|) / 10
//   6 near cells present / (3^d - 1)             7 ring cells present / (5^d - 3^d)
//   8 leaf box (its DOFs are points)             9 b / (sum of its children's b), 1 for a leaf
//  10 depth / 10          11 log2(1 + n_p) / 10  12 proxy radius / 5
//  13..15 zero
// |N| counts the level-start DOFs of the 3^d - 1 neighbour cells, |O| those of
// the ring at distance 2 (Sec. 3.2).
static void box_features(float *f, int dim, int kind, double eps, const ProxyParams &px, int depth, int b,
                         int nnear, int nring, int nnear_cells, int nring_cells, bool leaf, int child_sum) {
  const double n3 = dim == 3 ? 26.0 : 8.0, n5 = dim == 3 ? 98.0 : 16.0;
  f[0] = dim == 3 ? 1.f : 0.f;
  f[1] = (float)kind;
  f[2] = (float)(eps > 0 ? -log10(eps) / 10.0 : 1.6);
  f[3] = (float)(log2(1.0 + b) / 10.0);
  f[4] = (float)(log2(1.0 + nnear) / 10.0);
  f[5] = (float)(log2(1.0 + nring) / 10.0);
  f[6] = (float)(nnear_cells / n3);
  f[7] = (float)(nring_cells / n5);
  f[8] = leaf ? 1.f : 0.f;
  f[9] = leaf || child_sum <= 0 ? 1.f : (float)((double)b / child_sum);
  f[10] = (float)(depth / 10.0);
  f[11] = (float)(log2(1.0 + px.np) / 10.0);
  f[12] = (float)(px.radius / 5.0);
  for (int i = 13; i < MLP_NFEAT; i++) f[i] = 0.f;
}

// Proposed skeleton size from the predicted fraction k/b (NaN: k = b).
static int propose_k(int b, float frac) {
  if (!(frac == frac)) return b;
  const double f = std::min(1.0, std::max(0.0, (double)frac));
  return std::min(b, std::max(0, (int)std::lround(f * b)));
}

// Redundant DOFs to reserve storage for: the proposal's r plus a margin of
// max(4, b/8), at most b (NaN: no proposal, r = b).
static int reserve_rank(int b, float frac) {
  if (!(frac == frac)) return b;
  const int r = b - propose_k(b, frac) + std::max(4, (b + 7) / 8);
  return std::min(b, std::max(0, r));
}

template <typename T> static void run_factor(Factor<T> &F) {
  const int dim = F.dim;
  const int64_t n = F.n;
  const int np = F.nprob;
  cudaStream_t st = F.st;
  // points: tree order of every problem, concatenated (a single problem's
  // from the tree build's device arrays)
  if (F.dev_pts.have) {
    const double D = ldexp(1.0, -20);
    F.d_x.take(F.dev_pts.x);
    F.d_perm.take(F.dev_pts.perm);
    F.d_cell.alloc(sizeof(int) * 3 * (size_t)std::max<int64_t>(n, 1), st);
    F.d_off.alloc(sizeof(float) * 3 * (size_t)std::max<int64_t>(n, 1), st);
    points_setup(ptr<double>(F.d_x), ptr<int>(F.dev_pts.c20), n, dim, D, ptr<int>(F.d_cell), ptr<float>(F.d_off), st);
    check_launch("points setup");
    F.dev_pts.c20.release();  // stream-ordered: after the setup kernel
    F.P.x = ptr<double>(F.d_x);
    F.P.cell = ptr<int>(F.d_cell);
    F.P.off = ptr<float>(F.d_off);
    F.P.D = (float)D;
    F.P.dim = dim;
    F.P.wdof = nullptr;
  } else {
    std::vector<double> x((size_t)std::max<int64_t>(n, 1) * dim);
    std::vector<int64_t> perm(std::max<int64_t>(n, 1));
    std::vector<double> wd;
    std::vector<int> cell((size_t)3 * std::max<int64_t>(n, 1), 0);
    std::vector<float> off((size_t)3 * std::max<int64_t>(n, 1), 0.f);
    const double D = ldexp(1.0, -20);
    if (np > 1) wd.resize(std::max<int64_t>(n, 1));
    // split by problem and, within large problems, by DOF ranges
    std::vector<std::pair<int, int64_t>> chunks;
    for (int p = 0; p < np; p++)
      for (int64_t g0 = 0; g0 < F.trees[p].n; g0 += (int64_t)1 << 16) chunks.push_back({p, g0});
    HostPool::get().parallel_for((int64_t)chunks.size(), [&](int64_t ci) {
      const int p = chunks[ci].first;
      const HTree &Tp = F.trees[p];
      const int64_t o = F.pdof[p], g1 = std::min<int64_t>(Tp.n, chunks[ci].second + ((int64_t)1 << 16));
      for (int64_t g = chunks[ci].second; g < g1; g++) {
        perm[o + g] = o + Tp.perm[g];
        for (int d = 0; d < dim; d++) {
          const double v = Tp.x[g * dim + d];
          const int c = Tp.c20[g * dim + d];
          x[(o + g) * dim + d] = v;
          cell[3 * (o + g) + d] = c;
          off[3 * (o + g) + d] = (float)(v - (double)c * D);
        }
        if (np > 1) wd[o + g] = F.pw[p];
      }
    });
    upload(F.d_x, x, st);
    upload(F.d_perm, perm, st);
    upload(F.d_cell, cell, st);
    upload(F.d_off, off, st);
    if (np > 1) upload(F.d_wdof, wd, st);
    F.P.x = ptr<double>(F.d_x);
    F.P.cell = ptr<int>(F.d_cell);
    F.P.off = ptr<float>(F.d_off);
    F.P.D = (float)D;
    F.P.dim = dim;
    F.P.wdof = np > 1 ? ptr<double>(F.d_wdof) : nullptr;
  }
  {
    // direct-sum residual tiles: 256 targets of one problem against its sources
    std::vector<int64_t> ts, te, sb, se;
    for (int p = 0; p < np; p++)
      for (int64_t t0 = F.pdof[p]; t0 < F.pdof[p + 1]; t0 += 256) {
        ts.push_back(t0);
        te.push_back(std::min(t0 + 256, F.pdof[p + 1]));
        sb.push_back(F.pdof[p]);
        se.push_back(F.pdof[p + 1]);
      }
    F.mv_ntile = (int)ts.size();
    upload(F.d_mv_ts, ts, st);
    upload(F.d_mv_te, te, st);
    upload(F.d_mv_sb, sb, st);
    upload(F.d_mv_se, se, st);
  }
  F.d_err.alloc(sizeof(int), st);
  CK(cudaMemsetAsync(F.d_err.p, 0, sizeof(int), st));
  detect_grid(F);
  {
    // proxy surface template (Sec. 3.2): unit circle with n_p equispaced
    // angles in 2D, Fibonacci sphere with n_p points in 3D
    std::vector<double> u((size_t)3 * F.px.np, 0.0);
    for (int m = 0; m < F.px.np; m++) {
      if (dim == 2) {
        double th = 2.0 * kPi * (double)m / (double)F.px.np;
        u[3 * m] = cos(th);
        u[3 * m + 1] = sin(th);
      } else {
        double z = 1.0 - (2.0 * m + 1.0) / (double)F.px.np;
        double rr = sqrt(1.0 - z * z);
        double ph = (double)m * kPi * (3.0 - sqrt(5.0));
        u[3 * m] = rr * cos(ph);
        u[3 * m + 1] = rr * sin(ph);
        u[3 * m + 2] = z;
      }
    }
    std::vector<T> uT(u.begin(), u.end());  // the ID kernels read them in the factor's precision
    upload(F.d_proxy, uT, st);
  }

  F.maxdepth = 0;
  // box records: one per tree node of depths 2.. (RS-S); the hybrid has a
  // weak and a strong record per node of depths 2.. and a weak one at depth 1
  const bool hyb = (F.flags & RSS_FLAG_HYBRID) != 0;
  int nbox_total = 0;
  for (const HTree &Tp : F.trees) {
    F.maxdepth = std::max(F.maxdepth, Tp.maxdepth);
    for (int t = 2; t <= Tp.maxdepth; t++) nbox_total += (hyb ? 2 : 1) * (int)Tp.level[t].size();
    if (hyb && Tp.maxdepth >= 1) nbox_total += (int)Tp.level[1].size();
  }
  F.d_boxes.alloc(sizeof(FBox<T>) * std::max(nbox_total, 1), st);
  F.h_boxes.clear();
  F.phases.clear();

  // active DOFs of every problem (local tree-order ids, ascending)
  std::vector<std::vector<int64_t>> active(np);
  for (int p = 0; p < np; p++) {
    active[p].resize(F.trees[p].n);
    for (int64_t g = 0; g < F.trees[p].n; g++) active[p][g] = g;
  }
  DBuf d_dof_cell[2], d_dof_loc[2];
  std::unique_ptr<DLevel<T>> prevD;
  HLevel prevH;
  int prev_slot = 0;
  bool have_prev = false;

  // One problem without a rank proposal: the level lists are built on the
  // device from a device-resident active list (the host gets the cell and
  // pool counts and six ints per box); otherwise on the host (build_level).
  const bool dev_lv = np == 1 && !F.mlp && F.dev_pts.key.p != nullptr;
  DBuf d_act, d_act_next, lv_dk, lv_flag, lv_cpos, lv_cnt, lv_key, lv_grid, lv_psz, lv_tot, lv_node, lv_box;
  DBuf lv_sact, lv_k1, lv_v1, lv_hist;  // stable sorts of unsorted lists
  int64_t dev_na = 0;
  bool act_unsorted = false;  // the active list came out of a level in cell order, not ascending
  if (dev_lv) {
    dev_na = n;
    d_act.alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1), st);
    iota64(ptr<int64_t>(d_act), n, st);
    check_launch("active list");
  }
  auto build_level_dev = [&](const HTree &Tt, int t, DLevel<T> &D) {
    const int cbase = (F.flags & RSS_FLAG_COLOUR_2D) ? 2 : 3;  // colours per level, as below
    HLevel L;
    L.t = t;
    L.dim = dim;
    L.NB = dim == 2 ? 25 : 125;
    L.on_device = true;
    L.ndof = dev_na;
    const int64_t na = dev_na;
    grow(lv_dk, sizeof(uint64_t) * (size_t)na, st, 1);
    grow(lv_flag, sizeof(uint32_t) * (size_t)na, st, 1);
    grow(lv_cpos, sizeof(uint32_t) * (size_t)na, st, 1);
    grow(lv_cnt, 64, st, 1);
    auto sort_scratch = [&] {
      grow(lv_sact, sizeof(int64_t) * (size_t)na, st, 1);
      grow(lv_k1, sizeof(uint64_t) * (size_t)na, st, 1);
      grow(lv_v1, sizeof(int64_t) * (size_t)na, st, 1);
      grow(lv_hist, (size_t)sort_pairs_hist_bytes(na), st, 1);
    };
    if (act_unsorted) {  // the previous level left its survivors in cell order: ascending again
      sort_scratch();
      CK(cudaMemcpyAsync(lv_sact.p, d_act.p, sizeof(int64_t) * (size_t)na, cudaMemcpyDeviceToDevice, st));
      int bits = 1;
      while (bits < 62 && ((int64_t)1 << bits) < n) bits++;
      sort_pairs_u64(ptr<uint64_t>(lv_sact), ptr<int64_t>(d_act), ptr<uint64_t>(lv_k1), ptr<int64_t>(lv_v1),
                     ptr<uint32_t>(lv_hist), na, bits, st);
      act_unsorted = false;
    }
    CK(cudaMemsetAsync(lv_cnt.p, 0, 64, st));
    uint32_t *cnt = ptr<uint32_t>(lv_cnt);  // [0] cells, [1] unsorted
    level_gpu_keys(ptr<uint64_t>(F.dev_pts.key), ptr<int64_t>(d_act), na, dim * (20 - t), ptr<uint64_t>(lv_dk),
                   cnt + 1, st);
    level_gpu_runs(ptr<uint64_t>(lv_dk), na, ptr<uint32_t>(lv_flag), ptr<uint32_t>(lv_cpos), cnt, st);
    check_launch("level cells");
    uint32_t hc[2] = {0, 0};
    CK(cudaMemcpyAsync(hc, lv_cnt.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int64_t *act_lv = ptr<int64_t>(d_act);
    if (hc[1]) {
      // DOFs of leaves shallower than t are in their original order: a
      // stable sort of (key, DOF) groups them by cell, as the host build
      // does; the next level's list is made ascending again
      sort_scratch();
      CK(cudaMemcpyAsync(lv_sact.p, d_act.p, sizeof(int64_t) * (size_t)na, cudaMemcpyDeviceToDevice, st));
      sort_pairs_u64(ptr<uint64_t>(lv_dk), ptr<int64_t>(lv_sact), ptr<uint64_t>(lv_k1), ptr<int64_t>(lv_v1),
                     ptr<uint32_t>(lv_hist), na, dim * t, st);
      level_gpu_runs(ptr<uint64_t>(lv_dk), na, ptr<uint32_t>(lv_flag), ptr<uint32_t>(lv_cpos), cnt, st);
      check_launch("level sort");
      CK(cudaMemcpyAsync(hc, lv_cnt.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      act_lv = ptr<int64_t>(lv_sact);
      act_unsorted = true;
    }
    L.ncell = (int)hc[0];
    const int ncell = L.ncell;
    const int64_t len = (int64_t)ncell * L.NB;
    D.cell_dof_off.alloc(sizeof(int64_t) * (size_t)(ncell + 1), st);
    D.cell_dofs.alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(na, 1), st);
    D.cell_b.alloc(sizeof(int) * (size_t)std::max(ncell, 1), st);
    D.cell_coord.alloc(sizeof(int) * 3 * (size_t)std::max(ncell, 1), st);
    D.cell_nbr.alloc(sizeof(int) * (size_t)std::max<int64_t>(len, 1), st);
    D.pair_off.alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(len, 1), st);
    grow(lv_key, sizeof(uint64_t) * (size_t)std::max(ncell, 1), st, 1);
    grow(lv_psz, sizeof(unsigned long long) * (size_t)std::max<int64_t>(len, 1), st, 1);
    grow(lv_tot, 64, st, 1);
    CK(cudaMemsetAsync(lv_tot.p, 0, 64, st));  // pool total, bmax
    const int64_t side = (int64_t)1 << t;
    int64_t grid_cells = 1;
    for (int d = 0; d < dim; d++) grid_cells *= side;
    const bool use_grid = grid_cells <= ((int64_t)1 << 24);
    if (use_grid) {
      grow(lv_grid, sizeof(int) * (size_t)grid_cells, st, 1);
      CK(cudaMemsetAsync(lv_grid.p, 0xFF, sizeof(int) * (size_t)grid_cells, st));
    }
    // the tree's nodes of depth t, in the host order of build_level
    const std::vector<int> &nodes = Tt.level[t];
    const int nbox = (int)nodes.size();
    std::vector<int> ncoord((size_t)3 * std::max(nbox, 1), 0);
    for (int i = 0; i < nbox; i++)
      for (int d = 0; d < 3; d++) ncoord[3 * (size_t)i + d] = Tt.coord[3 * (size_t)nodes[i] + d];
    upload(lv_node, ncoord, st);
    grow(lv_box, sizeof(int) * 6 * (size_t)std::max(nbox, 1), st, 1);
    LevelGpu G;
    G.act = act_lv;
    G.na = na;
    G.dim = dim;
    G.NB = L.NB;
    G.side = (int)side;
    G.ncell = ncell;
    G.nbox = nbox;
    G.dk = ptr<uint64_t>(lv_dk);
    G.flag = ptr<uint32_t>(lv_flag);
    G.cpos = ptr<uint32_t>(lv_cpos);
    G.node_coord = ptr<int>(lv_node);
    G.grid = use_grid ? ptr<int>(lv_grid) : nullptr;
    G.cell_dof_off = ptr<int64_t>(D.cell_dof_off);
    G.cell_dofs = ptr<int64_t>(D.cell_dofs);
    G.pair_off = ptr<int64_t>(D.pair_off);
    G.cell_b = ptr<int>(D.cell_b);
    G.cell_coord = ptr<int>(D.cell_coord);
    G.cell_nbr = ptr<int>(D.cell_nbr);
    G.cell_key = ptr<uint64_t>(lv_key);
    G.psz = ptr<unsigned long long>(lv_psz);
    G.pool_total = ptr<unsigned long long>(lv_tot);
    G.bmax = reinterpret_cast<int *>(ptr<unsigned long long>(lv_tot) + 1);
    G.box_out = ptr<int>(lv_box);
    level_gpu_tables(G, st);
    check_launch("level tables");
    unsigned long long tot[2] = {0, 0};
    std::vector<int> bo((size_t)6 * std::max(nbox, 1));
    CK(cudaMemcpyAsync(tot, lv_tot.p, sizeof(tot), cudaMemcpyDeviceToHost, st));
    if (nbox > 0) CK(cudaMemcpyAsync(bo.data(), lv_box.p, sizeof(int) * 6 * (size_t)nbox, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    L.pool_elems = (int64_t)tot[0];
    L.bmax = (int)(tot[1] & 0xffffffffu);
    for (int i = 0; i < nbox; i++) {
      const int *o = &bo[6 * (size_t)i];
      if (o[0] < 0) continue;  // every DOF of the box has become inactive
      L.box_cell.push_back(o[0]);
      L.box_node.push_back(nodes[i]);
      L.box_colour.push_back(colour_of(&Tt.coord[3 * (size_t)nodes[i]], dim, cbase));
      L.box_b.push_back(o[1]);
      L.box_nj.push_back(o[2]);
      L.box_ring.push_back(o[3]);
      L.box_nnc.push_back(o[4]);
      L.box_nrc.push_back(o[5]);
    }
    if (cbase != 3) {  // as build_level: colour-major, node (Morton) order within a colour
      const int nb = (int)L.box_cell.size();
      std::vector<int> byn(nb), ord(nb);
      for (int q = 0; q < nb; q++) byn[q] = q;
      std::sort(byn.begin(), byn.end(), [&](int a, int b) { return L.box_node[a] < L.box_node[b]; });
      int ncol = 1;
      for (int d = 0; d < dim; d++) ncol *= cbase;
      std::vector<int> cstart(ncol + 1, 0);
      for (int q = 0; q < nb; q++) cstart[L.box_colour[q] + 1]++;
      for (int c = 0; c < ncol; c++) cstart[c + 1] += cstart[c];
      for (int q : byn) ord[cstart[L.box_colour[q]]++] = q;
      auto perm = [&](std::vector<int> &v) {
        std::vector<int> w(nb);
        for (int q = 0; q < nb; q++) w[q] = v[ord[q]];
        v.swap(w);
      };
      perm(L.box_cell), perm(L.box_node), perm(L.box_colour), perm(L.box_b), perm(L.box_nj), perm(L.box_ring);
      perm(L.box_nnc), perm(L.box_nrc);
    }
    return L;
  };

  auto assemble_pairs = [&](const HLevel &H, DLevel<T> &D, const LevelDev<T> *prev) {
    // one block per (cell, neighbour code at distance <= 2), enumerated on
    // the device from the level's tables; codes with no neighbour are empty
    const int64_t maxblk = (int64_t)H.bmax * H.bmax;
    AssembleList L{};
    L.nblock = H.ncell * H.NB;
    L.row_ids = L.col_ids = ptr<int64_t>(D.cell_dofs);
    L.cell_nbr = ptr<int>(D.cell_nbr);
    L.cell_b = ptr<int>(D.cell_b);
    L.cell_dof_off = ptr<int64_t>(D.cell_dof_off);
    L.pair_off = ptr<int64_t>(D.pair_off);
    L.NB = H.NB;
    int pi = F.prof.begin(KC_ASSEMBLE, st, 0, 0, 0, 2.0 * (double)H.pool_elems * sizeof(T), 0.0);
    launch_assemble<T>(L, ptr<T>(D.pool), prev, F.P, F.K, maxblk, st);
    F.prof.end(pi, st);
    check_launch("assemble");
  };

  // colours per level: 3^d (same-colour boxes share nothing) or the paper's 2^d
  const int cbase = (F.flags & RSS_FLAG_COLOUR_2D) ? 2 : 3;
  // symmetric storage: the kernels are symmetric, so G = E^T (Sec. 3.3) and
  // only E is kept
  const bool symm = (F.flags & RSS_FLAG_SYMMETRIC_STORAGE) != 0;
  std::unordered_map<int64_t, int> child_b;  // (problem, node) -> sum of its children's b
  DBuf gid, gel, gtri, gcnt;                 // per-phase ID and elimination scratch, grown as needed
  if (F.mlp) F.d_ovf_used.alloc(sizeof(unsigned long long), st);
  // stages: (depth, weak).  RS-S: the strong step at depths maxdepth .. 2.
  // RS-WS (Sec. 3.4, Algorithm 2): at each depth a weak pass over the boxes,
  // then the strong pass over what stays active, and a last weak pass at
  // depth 1.  The strong pass after a weak one rebuilds its level from the
  // weak pass's (same depth): the near-field blocks carry over.
  const bool hybrid = (F.flags & RSS_FLAG_HYBRID) != 0;
  std::vector<std::pair<int, int>> stages;
  for (int t = F.maxdepth; t >= (hybrid ? 1 : 2); t--) {
    if (hybrid) stages.push_back({t, 1});
    if (t >= 2) stages.push_back({t, 0});
  }
  for (const auto &stage : stages) {
    const int t = stage.first, weak = stage.second;
    double th0 = now_ms();
    // this depth's cells of every problem deep enough, merged
    HLevel H;
    H.t = t;
    H.dim = dim;
    H.NB = dim == 2 ? 25 : 125;
    std::vector<int> box_prob;
    std::vector<int> cell_base(np + 1, 0);
    std::unique_ptr<DLevel<T>> D(new DLevel<T>());
    if (dev_lv) {
      if (F.trees[0].maxdepth >= t && dev_na > 0) {
        H = build_level_dev(F.trees[0], t, *D);
        box_prob.assign(H.box_cell.size(), 0);
      }
    } else if (np == 1) {
      if (F.trees[0].maxdepth >= t && !active[0].empty()) {
        H = build_level(F.trees[0], t, active[0], cbase);
        box_prob.assign(H.box_cell.size(), 0);
      }
    } else {
      std::vector<HLevel> Hs(np);
      HostPool::get().parallel_for(np, [&](int64_t p) {
        if (F.trees[p].maxdepth >= t && !active[p].empty()) Hs[p] = build_level(F.trees[p], t, active[p], cbase);
      });
      size_t nc = 0, nd = 0, nbx = 0;
      for (int p = 0; p < np; p++) nc += Hs[p].ncell, nd += Hs[p].cell_dofs.size(), nbx += Hs[p].box_cell.size();
      H.cell_b.reserve(nc);
      H.cell_dof_off.reserve(nc + 1);
      H.cell_coord.reserve(3 * nc);
      H.cell_nbr.reserve(nc * H.NB);
      H.pair_off.reserve(nc * H.NB);
      H.cell_dofs.reserve(nd);
      H.box_cell.reserve(nbx);
      H.box_node.reserve(nbx);
      H.box_colour.reserve(nbx);
      box_prob.reserve(nbx);
      for (int p = 0; p < np; p++) {
        cell_base[p] = H.ncell;
        if (Hs[p].ncell == 0) continue;
        append_level(H, Hs[p], F.pdof[p], box_prob, p);
      }
    }
    if (np == 1) cell_base[0] = 0;
    cell_base[np] = H.ncell;
    if (H.cell_dof_off.empty()) H.cell_dof_off.push_back(0);
    if (!H.on_device) H.ndof = (int64_t)H.cell_dofs.size();
    if (H.box_cell.empty()) continue;  // no problem has boxes at this depth
    // colour-major order over all problems (stable: problem order within a colour)
    {
      const int nb0 = (int)H.box_cell.size();
      std::vector<int> ordr(nb0);
      for (int q = 0; q < nb0; q++) ordr[q] = q;
      std::stable_sort(ordr.begin(), ordr.end(), [&](int a, int b) { return H.box_colour[a] < H.box_colour[b]; });
      auto perm = [&](std::vector<int> &v) {
        if (v.empty()) return;
        std::vector<int> w(nb0);
        for (int q = 0; q < nb0; q++) w[q] = v[ordr[q]];
        v.swap(w);
      };
      perm(H.box_cell), perm(H.box_node), perm(H.box_colour), perm(box_prob);
      perm(H.box_b), perm(H.box_nj), perm(H.box_ring), perm(H.box_nnc), perm(H.box_nrc);
    }
    if (!H.on_device) {
      upload(D->cell_b, H.cell_b, st);
      upload(D->cell_dof_off, H.cell_dof_off, st);
      upload(D->cell_dofs, H.cell_dofs, st);
      upload(D->cell_coord, H.cell_coord, st);
      upload(D->cell_nbr, H.cell_nbr, st);
      upload(D->pair_off, H.pair_off, st);
    }
    D->pool.alloc((size_t)H.pool_elems * sizeof(T), st, 1);
    // active lists (every level-start DOF active, local order) and the
    // per-DOF maps of this level (-1 for DOFs in no cell), built on the device
    int slot = have_prev ? 1 - prev_slot : 0;
    {
      const size_t nd = (size_t)std::max<int64_t>(H.ndof, 1), nn = (size_t)std::max<int64_t>(n, 1);
      D->act_cnt.alloc(sizeof(int) * std::max(H.ncell, 1), st);
      D->act_idx.alloc(sizeof(int) * nd, st);
      if (H.ncell > 0)
        CK(cudaMemcpyAsync(D->act_cnt.p, D->cell_b.p, sizeof(int) * H.ncell, cudaMemcpyDeviceToDevice, st));
      if (d_dof_cell[slot].bytes < sizeof(int) * nn) {
        d_dof_cell[slot].alloc(sizeof(int) * nn, st);
        d_dof_loc[slot].alloc(sizeof(int) * nn, st);
      }
      CK(cudaMemsetAsync(d_dof_cell[slot].p, 0xFF, sizeof(int) * nn, st));
      CK(cudaMemsetAsync(d_dof_loc[slot].p, 0xFF, sizeof(int) * nn, st));
      launch_level_maps(H.ncell, ptr<int64_t>(D->cell_dof_off), ptr<int64_t>(D->cell_dofs), ptr<int>(D->act_idx),
                        ptr<int>(d_dof_cell[slot]), ptr<int>(d_dof_loc[slot]), st);
      check_launch("level_maps");
    }
    LevelDev<T> view = D->view(H, ptr<int>(d_dof_cell[slot]), ptr<int>(d_dof_loc[slot]));
    view.shared = cbase == 2;
    view.weak = weak;
    if (have_prev) {
      LevelDev<T> pv = prevD->view(prevH, ptr<int>(d_dof_cell[prev_slot]), ptr<int>(d_dof_loc[prev_slot]));
      assemble_pairs(H, *D, &pv);
    } else {
      assemble_pairs(H, *D, nullptr);
    }
    prevD.reset();  // stream-ordered free of the previous level

    // factor records of this level's boxes, and each box's features for the
    // rank proposal (sizes and geometry known before its ID)
    const int base = (int)F.h_boxes.size();
    const int nb = (int)H.box_cell.size();
    int njmax_lvl = 0, ring_max = 0;
    std::vector<int> njmaxv(nb), ringv(nb), bbox(nb);
    std::vector<float> fx((size_t)nb * MLP_NFEAT, 0.f);
    parallel_range(nb, 1024, [&](int64_t q0, int64_t q1) {
    for (int64_t q = q0; q < q1; q++) {
      int b, nj, ring, nnear_cells, nring_cells;
      if (H.on_device) {  // the device level build's per-box counts
        b = H.box_b[q];
        nj = H.box_nj[q];
        ring = H.box_ring[q];
        nnear_cells = H.box_nnc[q];
        nring_cells = H.box_nrc[q];
      } else {
        const int c = H.box_cell[q];
        b = H.cell_b[c];
        nj = b, nnear_cells = 0;
        int lim = dim == 3 ? 1 : 0;
        for (int dz = -lim; dz <= lim; dz++)
          for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
              if (!dx && !dy && !dz) continue;
              int nbc = H.cell_nbr[(size_t)c * H.NB + code5(dx, dy, dz, dim)];
              if (nbc >= 0) nj += H.cell_b[nbc], nnear_cells++;
            }
        // DOFs of the ring inside the proxy surface, bounded by level-start counts
        ring = 0, nring_cells = 0;
        int lim2 = dim == 3 ? 2 : 0;
        for (int dz = -lim2; dz <= lim2; dz++)
          for (int dy = -2; dy <= 2; dy++)
            for (int dx = -2; dx <= 2; dx++) {
              if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) != 2) continue;
              int nbc = H.cell_nbr[(size_t)c * H.NB + code5(dx, dy, dz, dim)];
              if (nbc >= 0) ring += H.cell_b[nbc], nring_cells++;
            }
      }
      bbox[q] = b;
      njmaxv[q] = weak ? b : nj;  // a weak step eliminates against J = S
      // rows of the ID matrix from inside the proxy surface: the ring, and
      // for a weak step the near cells too
      ringv[q] = weak ? ring + (nj - b) : ring;
      const HTree &Tp = F.trees[box_prob[q]];
      const int node = H.box_node[q];
      const bool leaf = !(Tp.count[node] > Tp.leaf && Tp.depth[node] < 20);
      int csum = 0;
      if (!leaf) {
        auto it = child_b.find(((int64_t)box_prob[q] << 32) | (uint32_t)node);
        csum = it == child_b.end() ? 0 : it->second;
      }
      box_features(&fx[(size_t)q * MLP_NFEAT], dim, F.K.kind, F.eps, F.px, t, b, nj - b, ring, nnear_cells,
                   nring_cells, leaf, csum);
    }
    });
    for (int q = 0; q < nb; q++) njmax_lvl = std::max(njmax_lvl, njmaxv[q]), ring_max = std::max(ring_max, ringv[q]);
    // reservations: full size (r = b, |J| = level-start count), or from the
    // proposed ranks plus margins
    std::vector<int> rres(nb), njres(njmaxv);
    for (int q = 0; q < nb; q++) rres[q] = bbox[q];
    if (F.mlp) {
      double tp0 = now_ms();
      DBuf d_fx, d_pr;
      upload(d_fx, fx, st);
      d_pr.alloc(sizeof(float) * std::max(nb, 1), st);
      mlp_forward(ptr<void>(F.mlp->wbf), ptr<float>(d_fx), nb, ptr<float>(d_pr), st);
      check_launch("mlp_forward");
      std::vector<float> pr(nb);
      CK(cudaMemcpyAsync(pr.data(), d_pr.p, sizeof(float) * nb, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      // proposed k per box; |J| at the box's turn counts the proposed
      // skeletons of neighbours eliminated in an earlier colour phase and all
      // level-start DOFs of the others
      std::vector<int> khat(nb), cell_box(H.ncell, -1);
      for (int q = 0; q < nb; q++) {
        const int b = H.cell_b[H.box_cell[q]];
        rres[q] = reserve_rank(b, pr[q]);
        khat[q] = propose_k(b, pr[q]);
        cell_box[H.box_cell[q]] = q;
      }
      for (int q = 0; q < nb; q++) {
        const int c = H.box_cell[q];
        int64_t nj = khat[q];
        const int lim = dim == 3 ? 1 : 0;
        for (int dz = -lim; dz <= lim; dz++)
          for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
              if (!dx && !dy && !dz) continue;
              const int nbc = H.cell_nbr[(size_t)c * H.NB + code5(dx, dy, dz, dim)];
              if (nbc < 0) continue;
              const int qn = cell_box[nbc];
              nj += (qn >= 0 && H.box_colour[qn] < H.box_colour[q]) ? khat[qn] : H.cell_b[nbc];
            }
        njres[q] = (int)std::min<int64_t>(njmaxv[q], nj + std::max<int64_t>(8, nj / 8));
      }
      F.prof.host(KC_HOST_LEVEL, now_ms() - tp0);
    }
    size_t sz_i64 = 0, sz_i32 = 0, sz_T = 0;
    for (int q = 0; q < nb; q++) {
      const size_t b = bbox[q], nj = njmaxv[q], rr = rres[q], njr = njres[q];
      sz_i64 += b + nj;
      sz_i32 += b + 2 * nj + b;
      sz_T += b * b / 4 + 1 + 2 * rr * rr + (symm ? 1 : 2) * njr * rr;
    }
    int64_t *p64 = (int64_t *)F.alloc_store(sz_i64 * sizeof(int64_t));
    int *p32 = (int *)F.alloc_store(sz_i32 * sizeof(int));
    T *pT = (T *)F.alloc_store(sz_T * sizeof(T));
    F.reserved_T += (int64_t)sz_T;
    for (int q = 0; q < nb; q++) {
      int c = H.box_cell[q], b = bbox[q], nj = njmaxv[q], rr = rres[q], njr = njres[q];
      FBox<T> fb{};
      fb.cell = c;
      fb.depth = t;
      fb.b = b;
      fb.njmax = nj;
      fb.rres = rr;
      fb.njres = njr;
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
      pT += (size_t)rr * rr;
      fb.Xi = pT;
      pT += (size_t)rr * rr;
      fb.E = pT;
      pT += (size_t)njr * rr;
      fb.G = symm ? nullptr : pT;  // symmetric storage: G = E^T is not kept
      if (!symm) pT += (size_t)njr * rr;
      F.h_boxes.push_back(fb);
    }
    F.feats.insert(F.feats.end(), fx.begin(), fx.end());
    // overflow space for boxes whose rank leaves more than the reservation
    Overflow<T> ovf{nullptr, nullptr, 0};
    if (F.mlp) {
      int64_t cap = (int64_t)(sz_T / 16) + 2 * (2 * (int64_t)H.bmax * H.bmax + 2 * (int64_t)njmax_lvl * H.bmax) + 64;
      ovf.base = (T *)F.alloc_store((size_t)cap * sizeof(T));
      ovf.cap = cap;
      ovf.used = ptr<unsigned long long>(F.d_ovf_used);
      F.reserved_T += cap;
      CK(cudaMemsetAsync(F.d_ovf_used.p, 0, sizeof(unsigned long long), st));
    }
    staged_h2d(ptr<FBox<T>>(F.d_boxes) + base, F.h_boxes.data() + base, sizeof(FBox<T>) * nb, st);
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
    const bool large = (F.flags & RSS_FLAG_LARGE_BOX_PATH) != 0;
    int PR = H.bmax <= 80 ? 128 : 64;
    int64_t idb = id_region_bytes<T>(H.bmax, PR);
    bool id_smem = idb <= 200 * 1024 && !large;
    int64_t id_stride = (idb + sizeof(T) - 1) / sizeof(T) + 32;
    // boxes wider than 512 (3D upper levels at small eps): the general ID
    // over up to 32 CTAs per box (about two CTAs per SM over the largest
    // phase), each with its own workspace, at most 8 GB of them
    int kid_ctas = 1;
    if (H.bmax > 512 && !id_smem && !large) {
      const int mp = std::max(maxphase, 1);
      kid_ctas = std::min(32, (304 + mp - 1) / mp);
      while (kid_ctas > 1 && (double)id_stride * sizeof(T) * mp * kid_ctas > 8e9) kid_ctas /= 2;
    }
    if (!id_smem) grow(gid, (size_t)id_stride * sizeof(T) * std::max(maxphase, 1) * kid_ctas, st, 1);
    int64_t el_stride = 2 * (int64_t)njmax_lvl * H.bmax + 32 + elim_ws_elems<T>(H.bmax);
    grow(gel, (size_t)el_stride * sizeof(T) * std::max(maxphase, 1), st, 1);
    // the multi-CTA ID's triangle slots (8 CTAs per box of the largest
    // phase, 16 for boxes wider than 256) and tree-node counters
    IdMultiScratch ims{};
    if (H.bmax <= 512 && !large) {
      const int64_t se = H.bmax <= 64 ? 64 * 65 : H.bmax <= 128 ? 128 * 129 : (int64_t)H.bmax * (H.bmax + 1);
      const int64_t slots = (H.bmax > 256 ? 16 : 8) * (int64_t)std::max(maxphase, 1);
      grow(gtri, (size_t)(slots * se) * sizeof(T), st, 1);
      grow(gcnt, sizeof(int) * (size_t)slots * 8, st, 1);
      CK(cudaMemsetAsync(gcnt.p, 0, sizeof(int) * (size_t)slots * 8, st));
      ims = IdMultiScratch{gtri.p, se, slots, ptr<int>(gcnt)};
    } else if (kid_ctas > 1) {
      const int64_t slots = (int64_t)kid_ctas * std::max(maxphase, 1);
      grow(gcnt, sizeof(int) * (size_t)slots * 8, st, 1);
      CK(cudaMemsetAsync(gcnt.p, 0, sizeof(int) * (size_t)slots * 8, st));
      ims = IdMultiScratch{nullptr, 0, slots, ptr<int>(gcnt), kid_ctas};
    }
    set_id_multi(ims);
    F.prof.host(KC_HOST_LEVEL, now_ms() - th0);
    for (auto &p : ph) {
      const int *bl = ptr<int>(d_list) + p.first;
      auto id_launch = [&] {
        launch_id<T>(view, ptr<FBox<T>>(F.d_boxes), bl, p.second, large ? -H.bmax : H.bmax, ring_max, F.P, F.K, F.px,
                     ptr<T>(F.d_proxy), F.eps, ptr<T>(gid), id_stride, id_smem, st, ptr<int>(F.d_err));
      };
      int pi = F.prof.begin(KC_ID, st, base + p.first, p.second);
      tuned_id_launch(F, large ? -H.bmax : H.bmax, p.second, id_launch);
      check_launch("id");
      F.prof.end(pi, st);
      pi = F.prof.begin(KC_ELIM, st, base + p.first, p.second);
      auto elim_launch = [&] {
        launch_elim<T>(view, ptr<FBox<T>>(F.d_boxes), bl, p.second, large ? -H.bmax : H.bmax, ptr<T>(gel), el_stride,
                       ovf, st, ptr<int>(F.d_err), njmax_lvl);
      };
      tuned_elim_launch(F, large ? -H.bmax : H.bmax, p.second, elim_launch);
      check_launch("elim");
      F.prof.end(pi, st);
      pi = F.prof.begin(KC_SCHUR, st, base + p.first, p.second);
      if constexpr (std::is_same<T, float>::value) {
        if (!(F.flags & RSS_FLAG_NO_TENSOR_CORES))
          launch_schur_tc(view, ptr<FBox<T>>(F.d_boxes), bl, p.second, njmax_lvl, ptr<T>(gel), el_stride, st,
                          ptr<int>(F.d_err));
        else
          launch_schur<T>(view, ptr<FBox<T>>(F.d_boxes), bl, p.second, njmax_lvl, ptr<T>(gel), el_stride, st);
      } else {
        launch_schur<T>(view, ptr<FBox<T>>(F.d_boxes), bl, p.second, njmax_lvl, ptr<T>(gel), el_stride, st);
      }
      check_launch("schur");
      F.prof.end(pi, st);
      F.phases.push_back({base + p.first, p.second, H.bmax, large ? -njmax_lvl : njmax_lvl, 0, 0, cbase == 2});
    }
    set_id_multi(IdMultiScratch{});
    // ranks of this level -> active DOFs of the next
    CK(cudaMemcpyAsync(F.h_boxes.data() + base, ptr<FBox<T>>(F.d_boxes) + base, sizeof(FBox<T>) * nb,
                       cudaMemcpyDeviceToHost, st));
    std::vector<int> ac(H.on_device ? 0 : H.ncell), ai(H.on_device ? 0 : H.cell_dofs.size());
    uint32_t next_na = 0;
    if (H.on_device) {  // the next level's active list, compacted on the device
      d_act_next.alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(dev_na, 1), st);
      grow(lv_cpos, sizeof(uint32_t) * (size_t)std::max(H.ncell, 1), st, 1);
      level_gpu_next_active(H.ncell, ptr<int64_t>(D->cell_dof_off), ptr<int64_t>(D->cell_dofs), ptr<int>(D->act_cnt),
                            ptr<int>(D->act_idx), ptr<uint32_t>(lv_cpos), ptr<uint32_t>(lv_cnt),
                            ptr<int64_t>(d_act_next), st);
      check_launch("next active list");
      CK(cudaMemcpyAsync(&next_na, lv_cnt.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    } else {
      CK(cudaMemcpyAsync(ac.data(), D->act_cnt.p, sizeof(int) * H.ncell, cudaMemcpyDeviceToHost, st));
      if (!ai.empty())
        CK(cudaMemcpyAsync(ai.data(), D->act_idx.p, sizeof(int) * ai.size(), cudaMemcpyDeviceToHost, st));
    }
    unsigned long long ovf_used = 0;
    if (F.mlp) CK(cudaMemcpyAsync(&ovf_used, F.d_ovf_used.p, sizeof(ovf_used), cudaMemcpyDeviceToHost, st));
    double tw0 = now_ms();
    int e = check_err(F.d_err, st);
    F.prof.host(KC_HOST_WAIT, now_ms() - tw0);
    prof_collect(F);
    if (e == DERR_NUMERIC) throw Fail{RSS_ENUMERIC, "zero pivot in the LU of a redundant block"};
    if (e == DERR_CAPACITY) throw Retry{};
    if (e) throw Fail{RSS_ECUDA, "device-side consistency check failed"};
    F.ovf_used += (int64_t)ovf_used;
    // ranks of this level: storage they need, and child sizes for the next level's features
    child_b.clear();
    for (int q = 0; q < nb; q++) {
      const FBox<T> &fb = F.h_boxes[base + q];
      F.used_T += (int64_t)fb.k * fb.r + 2 * (int64_t)fb.r * fb.r + (symm ? 1 : 2) * (int64_t)fb.nj * fb.r;
      const HTree &Tp = F.trees[box_prob[q]];
      const int par = Tp.parent[H.box_node[q]];
      if (par >= 0) child_b[((int64_t)box_prob[q] << 32) | (uint32_t)par] += fb.b;
    }
    double ta0 = now_ms();
    if (H.on_device) {
      dev_na = (int64_t)next_na;
      std::swap(d_act.p, d_act_next.p);
      std::swap(d_act.bytes, d_act_next.bytes);
      std::swap(d_act.st, d_act_next.st);
    } else {
    // each cell's active DOFs at its offset in the problem's list (an
    // exclusive scan of the counts), filled in parallel over cells
    std::vector<int64_t> aoff(H.ncell + 1, 0);
    for (int c = 0; c < H.ncell; c++) aoff[c + 1] = aoff[c] + ac[c];
    for (int p = 0; p < np; p++)
      if (cell_base[p + 1] > cell_base[p]) active[p].resize(aoff[cell_base[p + 1]] - aoff[cell_base[p]]);
    std::vector<int> cell_prob(H.ncell);
    for (int p = 0; p < np; p++)
      for (int c = cell_base[p]; c < cell_base[p + 1]; c++) cell_prob[c] = p;
    parallel_range(H.ncell, 256, [&](int64_t c0, int64_t c1) {
      for (int64_t c = c0; c < c1; c++) {
        const int p = cell_prob[c];
        int64_t *dst = active[p].data() + (aoff[c] - aoff[cell_base[p]]);
        for (int q = 0; q < ac[c]; q++) dst[q] = H.cell_dofs[H.cell_dof_off[c] + ai[H.cell_dof_off[c] + q]] - F.pdof[p];
      }
    });
    HostPool::get().parallel_for(np, [&](int64_t p) {
      if (cell_base[p + 1] == cell_base[p]) return;
      std::vector<int64_t> &act = active[p];
      if (!std::is_sorted(act.begin(), act.end())) std::sort(act.begin(), act.end());
    });
    }
    F.prof.host(KC_HOST_LEVEL, now_ms() - ta0);
    prevD = std::move(D);
    prevH = std::move(H);
    prev_slot = slot;
    have_prev = true;
  }

  // solve-sweep work items: every box with r > 0 in chunks of SWEEP_CHUNK rows of J
  {
    std::vector<int> wb, wc;
    std::vector<int64_t> poff(F.h_boxes.size() + 1, 0);
    for (size_t q = 0; q < F.h_boxes.size(); q++) {
      const FBox<T> &b = F.h_boxes[q];
      const int nch = std::max(1, (b.nj + SWEEP_CHUNK - 1) / SWEEP_CHUNK);
      poff[q + 1] = poff[q] + (b.r > 0 ? (int64_t)nch * b.r * 4 : 0);
    }
    for (Phase &p : F.phases) {
      p.wfirst = (int)wb.size();
      for (int q = p.first; q < p.first + p.count; q++) {
        const FBox<T> &b = F.h_boxes[q];
        if (b.r == 0) continue;
        const int nch = std::max(1, (b.nj + SWEEP_CHUNK - 1) / SWEEP_CHUNK);
        for (int c = 0; c < nch; c++) wb.push_back(q), wc.push_back(c);
      }
      p.wcount = (int)wb.size() - p.wfirst;
    }
    upload(F.d_wbox, wb, st);
    upload(F.d_wchunk, wc, st);
    upload(F.d_poff, poff, st);
    F.d_wcnt.alloc(sizeof(int) * std::max<size_t>(F.h_boxes.size(), 1), st);
    CK(cudaMemsetAsync(F.d_wcnt.p, 0, sizeof(int) * std::max<size_t>(F.h_boxes.size(), 1), st));
    F.d_pbuf.alloc(sizeof(T) * std::max<int64_t>(poff.back(), 1), st);
  }

  // top blocks: every problem's DOFs still active (Sec. 3.3.3), dense LU
  if (dev_lv) {  // the active list after the last level, for the top block
    active[0].resize(dev_na);
    if (dev_na > 0)
      CK(cudaMemcpyAsync(active[0].data(), d_act.p, sizeof(int64_t) * dev_na, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (act_unsorted) std::sort(active[0].begin(), active[0].end());
  }
  std::vector<int64_t> top;
  F.h_tn.assign(np, 0);
  F.h_toff.assign(np + 1, 0);
  F.h_loff.assign(np + 1, 0);
  for (int p = 0; p < np; p++) {
    F.h_tn[p] = (int)active[p].size();
    F.h_toff[p + 1] = F.h_toff[p] + F.h_tn[p];
    F.h_loff[p + 1] = F.h_loff[p] + (int64_t)F.h_tn[p] * F.h_tn[p];
    for (int64_t g : active[p]) top.push_back(g + F.pdof[p]);
  }
  F.ntop = (int)top.size();
  upload(F.d_top, top, st);
  upload(F.d_tn, F.h_tn, st);
  upload(F.d_toff, F.h_toff, st);
  upload(F.d_loff, F.h_loff, st);
  F.d_topLU.alloc((size_t)F.h_loff[np] * sizeof(T) + 16, st);
  F.d_toppiv.alloc((size_t)F.ntop * sizeof(int) + 16, st);
  F.factor_bytes += (int64_t)F.h_loff[np] * sizeof(T) + (int64_t)F.ntop * (sizeof(int) + 8);
  if (F.ntop > 0) {
    std::vector<int> nr(F.h_tn.begin(), F.h_tn.end());
    DBuf d_nr;
    upload(d_nr, nr, st);
    // the dense LU works on row-major matrices: assemble the transpose layout
    AssembleList L{np, ptr<int64_t>(F.d_toff), ptr<int64_t>(F.d_toff), ptr<int64_t>(F.d_loff), ptr<int>(d_nr),
                   ptr<int>(d_nr), ptr<int64_t>(F.d_top), ptr<int64_t>(F.d_top), 1};
    int maxt = *std::max_element(F.h_tn.begin(), F.h_tn.end());
    if (have_prev) {
      LevelDev<T> pv = prevD->view(prevH, ptr<int>(d_dof_cell[prev_slot]), ptr<int>(d_dof_loc[prev_slot]));
      launch_assemble<T>(L, ptr<T>(F.d_topLU), &pv, F.P, F.K, (int64_t)maxt * maxt, st);
    } else {
      launch_assemble<T>(L, ptr<T>(F.d_topLU), nullptr, F.P, F.K, (int64_t)maxt * maxt, st);
    }
    check_launch("assemble top");
    double fl = 0;
    for (int tn : F.h_tn) fl += 2.0 / 3.0 * (double)tn * tn * tn;
    int pi = F.prof.begin(KC_TOPLU, st, 0, 0, 0, 2.0 * (double)F.h_loff[np] * sizeof(T), fl);
    DBuf d_panel;  // column-major copy of the current panel
    if (np == 1) {
      d_panel.alloc((size_t)F.ntop * 32 * sizeof(T) + 32 * sizeof(int), st, 1);  // + the interchanges
      launch_dense_lu<T>(ptr<T>(F.d_topLU), F.ntop, ptr<int>(F.d_toppiv), ptr<T>(d_panel), st, ptr<int>(F.d_err));
    } else
      launch_lu_batched<T>(ptr<T>(F.d_topLU), ptr<int64_t>(F.d_loff), ptr<int>(F.d_toppiv), ptr<int64_t>(F.d_toff),
                           ptr<int>(F.d_tn), np, st, ptr<int>(F.d_err));
    check_launch("top lu");
    if (np == 1 && F.ntop <= 1024) {
      // the solves multiply by U^{-1} L^{-1} instead of two triangular sweeps
      F.d_topinv.alloc((size_t)F.ntop * F.ntop * sizeof(T), st);
      F.factor_bytes += (int64_t)F.ntop * F.ntop * sizeof(T);
      launch_top_inverse<T>(ptr<T>(F.d_topLU), F.ntop, ptr<T>(F.d_topinv), st);
      check_launch("top inverse");
    }
    F.prof.end(pi, st);
  }
  prevD.reset();
  if (F.async()) {  // the top block's LU runs on; its error flag is read by a later call
    defer_err(F);
    return;
  }
  int e = check_err(F.d_err, st);
  prof_collect(F);
  if (e == DERR_NUMERIC) throw Fail{RSS_ENUMERIC, "zero pivot in the top block"};
  if (e) throw Fail{RSS_ECUDA, "device-side consistency check failed"};
}

}  // namespace rss

struct rss_factorization {
  uint32_t magic = rss::MAGIC_FACTOR;
  std::unique_ptr<rss::FactorBase> impl;
};

struct rss_mlp {
  uint32_t magic = rss::MAGIC_MLP;
  std::unique_ptr<rss::MlpModel> impl;
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

// One phase of a sweep: the chunked solve kernels when they apply, else the
// one-CTA-per-box kernel (apply sweeps, more than four right-hand sides, the
// forced large-box path).
template <typename T>
static void sweep_phase(const Factor<T> &F, int mode, const Phase &p, T *v, int nrhs, cudaStream_t st) {
  const bool solve = mode == SWEEP_SOLVE_FWD || mode == SWEEP_SOLVE_BWD;
  if (solve && nrhs <= 4 && p.njmax >= 0 && sweep_chunk_smem(p.bmax, nrhs, sizeof(T)) <= (size_t)(200 << 10)) {
    launch_sweep_chunks<T>(mode, ptr<FBox<T>>(F.d_boxes), ptr<int>(F.d_wbox) + p.wfirst, ptr<int>(F.d_wchunk) + p.wfirst,
                           p.wcount, v, nrhs, p.bmax, ptr<int>(F.d_wcnt), ptr<T>(F.d_pbuf), ptr<int64_t>(F.d_poff), st,
                           p.shared);
    return;
  }
  launch_sweep<T>(mode, ptr<FBox<T>>(F.d_boxes), p.first, p.count, v, nrhs, p.bmax, p.njmax, st, p.shared);
}

// Every launch of one application of F (Eq. 3.10) or F^{-1} (Eq. 3.11) on
// `st`: permute into tree order, forward sweeps over the phases, the top
// blocks, backward sweeps, permute back.  Per-launch profiling when `prof`.
template <typename T>
static void enqueue_sweeps(const Factor<T> &F, const double *in, double *out, T *v, int nrhs, bool solve,
                           cudaStream_t st, bool prof) {
  Prof &P = F.prof;
  auto begin = [&](int cls, int first, int count, int nr, double bytes = 0.0, double flops = 0.0) {
    return prof ? P.begin(cls, st, first, count, nr, bytes, flops) : -1;
  };
  auto end = [&](int pi) {
    if (prof) P.end(pi, st);
  };
  const double sz = sizeof(T);
  int pi = begin(KC_PERMUTE, 0, 0, 0, (double)F.n * nrhs * (8.0 + sz + 8.0));
  launch_permute<T>(0, ptr<int64_t>(F.d_perm), in, v, nullptr, F.n, nrhs, st);
  end(pi);
  const int fwd = solve ? SWEEP_SOLVE_FWD : SWEEP_APPLY_FWD, bwd = solve ? SWEEP_SOLVE_BWD : SWEEP_APPLY_BWD;
  for (const Phase &p : F.phases) {
    pi = begin(KC_SWEEP, p.first, p.count, nrhs);
    sweep_phase<T>(F, fwd, p, v, nrhs, st);
    end(pi);
  }
  double nt = F.ntop;
  pi = begin(KC_TOP, 0, 0, 0, nt * nt * sz + 2.0 * nt * nrhs * sz, 2.0 * nt * nt * nrhs);
  launch_top<T>(solve ? 0 : 1, ptr<T>(F.d_topLU), ptr<int64_t>(F.d_loff), ptr<int>(F.d_toppiv), ptr<int64_t>(F.d_top),
                ptr<int64_t>(F.d_toff), ptr<int>(F.d_tn), F.nprob, F.ntop, v, nrhs, ptr<T>(F.d_topwork), st,
                F.d_topinv.p ? ptr<T>(F.d_topinv) : nullptr);
  end(pi);
  for (auto it = F.phases.rbegin(); it != F.phases.rend(); ++it) {
    pi = begin(KC_SWEEP, it->first, it->count, nrhs);
    sweep_phase<T>(F, bwd, *it, v, nrhs, st);
    end(pi);
  }
  pi = begin(KC_PERMUTE, 0, 0, 0, (double)F.n * nrhs * (8.0 + sz + 8.0));
  launch_permute<T>(1, ptr<int64_t>(F.d_perm), nullptr, v, out, F.n, nrhs, st);
  end(pi);
}

// The solve's launch sequence for nrhs <= 4 as a CUDA graph (reading g_in,
// writing g_out), captured on a private stream and replayed on the factor's
// stream.  It is captured right after the first (uncaptured) solve with this
// nrhs, which has set the kernel attributes and loaded the kernels; the GPU
// is still running that solve while the host captures.  Rebuilt when the
// working vectors are reallocated.
template <typename T> static void capture_solve_graph(const Factor<T> &F, int nrhs) {
  auto &g = F.sgraph[nrhs];
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  const size_t nb = sizeof(double) * (size_t)std::max<int64_t>(F.n, 1) * 4;
  grow(F.g_in, nb, F.st);
  grow(F.g_out, nb, F.st);
  T *v = ptr<T>(F.d_work);
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const long long l0 = launches_total();
    enqueue_sweeps(F, ptr<double>(F.g_in), ptr<double>(F.g_out), v, nrhs, true, cs, false);
    g.kernels = (int)(launches_total() - l0);
    count_launch(-g.kernels);  // captured, not launched
    e = cudaStreamEndCapture(cs, &graph);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g.exec = nullptr;
    throw Fail{RSS_ECUDA, std::string("capturing the solve sweeps: ") + cudaGetErrorString(e)};
  }
  g.gen = F.work_gen;
}

template <typename T>
static void do_sweeps(const Factor<T> &F, const double *in, double *out, int nrhs, bool solve, bool sync = true) {
  cudaStream_t st = F.st;
  ensure_work(F, nrhs);
  T *v = ptr<T>(F.d_work);
  const bool graphed = solve && F.use_graphs && nrhs <= 4 && F.n > 0;
  if (graphed && !(F.sgraph[nrhs].exec && F.sgraph[nrhs].gen == F.work_gen)) {
    enqueue_sweeps(F, in, out, v, nrhs, solve, st, F.prof.on);
    check_launch("sweeps");
    capture_solve_graph(F, nrhs);
  } else if (graphed) {
    cudaGraphExec_t ge = F.sgraph[nrhs].exec;
    const size_t nb = sizeof(double) * (size_t)F.n * nrhs;
    int pi = F.prof.begin(KC_SWEEP, st, 0, (int)F.h_boxes.size(), nrhs);
    CK(cudaMemcpyAsync(F.g_in.p, in, nb, cudaMemcpyDeviceToDevice, st));
    CK(cudaGraphLaunch(ge, st));
    CK(cudaMemcpyAsync(out, F.g_out.p, nb, cudaMemcpyDeviceToDevice, st));
    F.prof.end(pi, st);
    count_launch(F.sgraph[nrhs].kernels);
  } else {
    enqueue_sweeps(F, in, out, v, nrhs, solve, st, F.prof.on);
    check_launch("sweeps");
  }
  if (sync && !F.async()) {
    CK(cudaStreamSynchronize(st));
    prof_collect(F);
  }
}

template <typename T> static void apply_A_impl(const Factor<T> &F, const double *x, double *y, int nrhs, bool f32);

// y = A x in FP64 (f32: the kernel sums or the FFT convolution in FP32, for
// the inner GMRES of the refinement; y is FP64 either way)
template <typename T> static void apply_A(const Factor<T> &F, const double *x, double *y, int nrhs, bool f32 = false) {
  // FP64 flops of the FFT operator (the work of this class): per pair of
  // right-hand sides a forward and an inverse transform over the lines the
  // zero padding leaves (along axis a, the lines whose coordinates before a
  // span L and after a span s), 5 L log2 L flops a line, and the pointwise
  // product (6 flops per frequency)
  double fl = 0.0;
  if (F.grid_side > 0) {
    const double s = F.grid_side, L = 2.0 * F.grid_side;
    double lines = 0.0, vol = 1.0;
    for (int a = 0; a < F.dim; a++) {
      double l = 1.0;
      for (int d = 0; d < F.dim; d++)
        if (d != a) l *= d < a ? L : s;
      lines += l;
      vol *= L;
    }
    fl = (double)((nrhs + 1) / 2) * (2.0 * lines * 5.0 * L * std::log2(L) + 6.0 * vol);
  }
  int pi = F.prof.begin(f32 ? KC_INNER_OP : KC_REFINE_OP, F.st, 0, 0, nrhs, 0.0, fl);
  apply_A_impl(F, x, y, nrhs, f32);
  F.prof.end(pi, F.st);
}

template <typename T> static void apply_A_impl(const Factor<T> &F, const double *x, double *y, int nrhs, bool f32) {
  if (F.grid_side > 0) {
    if (!F.grid_ready) {
      GridOp &G = F.G;
      G.dim = F.dim;
      G.s = F.grid_side;
      G.L = 2 * F.grid_side;
      G.logL = 0;
      while ((1 << G.logL) < G.L) G.logL++;
      G.n = F.n;
      G.h = 1.0 / F.grid_side;
      G.kind = F.K.kind;
      G.w = F.K.w;
      G.diag = F.K.diag;
      int64_t tot = 1;
      for (int d = 0; d < G.dim; d++) tot *= G.L;
      if (!F.grid_index.empty()) upload(F.g_gidx, F.grid_index, F.st);  // else detected on the device
      F.g_C.alloc(sizeof(double2) * tot, F.st);
      F.g_X.alloc(sizeof(double2) * tot, F.st);
      F.g_tw.alloc(sizeof(double2) * G.L, F.st);
      G.gidx = ptr<int64_t>(F.g_gidx);
      G.C = ptr<double2>(F.g_C);
      G.X = ptr<double2>(F.g_X);
      G.tw = ptr<double2>(F.g_tw);
      grid_op_setup(G, F.st);
      check_launch("grid operator setup");
      F.grid_ready = true;
    }
    if (f32 && !F.grid_f32_ready) {
      GridOp &G = F.G;
      int64_t tot = 1;
      for (int d = 0; d < G.dim; d++) tot *= G.L;
      F.g_Cf.alloc(sizeof(float2) * tot, F.st);
      F.g_Xf.alloc(sizeof(float2) * tot, F.st);
      F.g_twf.alloc(sizeof(float2) * G.L, F.st);
      G.Cf = ptr<float2>(F.g_Cf);
      G.Xf = ptr<float2>(F.g_Xf);
      G.twf = ptr<float2>(F.g_twf);
      grid_op_setup_f32(G, F.st);
      check_launch("grid operator setup (FP32)");
      F.grid_f32_ready = true;
    }
    grid_op_apply(F.G, x, y, nrhs, F.st, f32);
  } else if (f32) {
    launch_matvec_f32(F.P, F.K, ptr<int64_t>(F.d_perm), x, y, F.n, nrhs, F.mv_ntile, ptr<int64_t>(F.d_mv_ts),
                      ptr<int64_t>(F.d_mv_te), ptr<int64_t>(F.d_mv_sb), ptr<int64_t>(F.d_mv_se), F.st);
  } else {
    launch_matvec(ptr<double>(F.d_x), F.dim, F.K, F.P.wdof, ptr<int64_t>(F.d_perm), x, y, F.n, nrhs, F.mv_ntile,
                  ptr<int64_t>(F.d_mv_ts), ptr<int64_t>(F.d_mv_te), ptr<int64_t>(F.d_mv_sb), ptr<int64_t>(F.d_mv_se),
                  F.st);
  }
  check_launch("residual operator");
}

// GMRES-based iterative refinement (Carson & Higham): FP64 residuals with
// the exact operator, each correction from restarted, right-preconditioned
// FGMRES in FP64 whose preconditioner is the factor's solve (FP32 for the
// mixed factor).  For the mixed factor the operator products inside FGMRES
// are FP32 (kernel sums or FFT convolution accurate to FP32 rounding, FP64
// vectors): the correction only needs relative accuracy well below 1, and
// the next FP64 residual measures what it achieved.  All right-hand sides
// advance in lock step.
template <typename T>
static bool refine(const Factor<T> &F, const double *b, double *x, int nrhs, double tol, int maxit, int *iters,
                   double *relres) {
  cudaStream_t st = F.st;
  const int64_t n = F.n, nn = n * nrhs;
  const int m = 10;
  DBuf r, w, V, Z, part, dres;
  r.alloc(sizeof(double) * nn, st);
  w.alloc(sizeof(double) * nn, st);
  V.alloc(sizeof(double) * nn * (m + 1), st);
  Z.alloc(sizeof(double) * nn * m, st);
  part.alloc(sizeof(double) * (m + 1) * nrhs * 240, st);
  dres.alloc(sizeof(double) * (m + 1) * nrhs * 2, st);
  double *pr = ptr<double>(r), *pw = ptr<double>(w), *pV = ptr<double>(V), *pZ = ptr<double>(Z);
  double *dd = ptr<double>(dres), *dc = dd + (m + 1) * nrhs;
  std::vector<double> h((m + 1) * nrhs), h2((m + 1) * nrhs);
  auto dots = [&](const double *Vb, int nv, const double *vec, std::vector<double> &out) {
    multidot(Vb, nn, nv, vec, n, nrhs, ptr<double>(part), dd, st);
    check_launch("multidot");
    out.resize((size_t)nv * nrhs);
    CK(cudaMemcpyAsync(out.data(), dd, sizeof(double) * nv * nrhs, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  };
  auto comb = [&](double *y, double alpha, const double *Vb, int nv, const std::vector<double> &coef) {
    staged_h2d(dc, coef.data(), sizeof(double) * nv * nrhs, st);
    combine(y, alpha, Vb, nn, nv, dc, n, nrhs, st);
    check_launch("combine");
  };
  // x0 = F^{-1} b
  do_sweeps(F, b, x, nrhs, true, false);
  std::vector<double> bn;
  dots(b, 1, b, bn);
  for (auto &v : bn) v = v > 0 ? sqrt(v) : 1.0;
  int inner = 0;
  double rel = 0;
  bool ok = false;
  for (int outer = 0; outer <= maxit; outer++) {
    apply_A(F, x, pw, nrhs);
    CK(cudaMemcpyAsync(pr, b, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
    comb(pr, 1.0, pw, 1, std::vector<double>(nrhs, -1.0));
    std::vector<double> rn;
    dots(pr, 1, pr, rn);
    rel = 0;
    for (int c = 0; c < nrhs; c++) {
      rn[c] = sqrt(std::max(rn[c], 0.0));
      rel = std::max(rel, rn[c] / bn[c]);
    }
    if (rel <= tol) {
      ok = true;
      break;
    }
    if (outer == maxit) break;
    // FGMRES(m) for A d = r, right-preconditioned by F^{-1}
    std::vector<double> inv(nrhs);
    for (int c = 0; c < nrhs; c++) inv[c] = rn[c] > 0 ? 1.0 / rn[c] : 0.0;
    CK(cudaMemsetAsync(pV, 0, sizeof(double) * nn, st));
    comb(pV, 0.0, pr, 1, inv);
    std::vector<double> H((size_t)nrhs * (m + 1) * m, 0.0), g((size_t)nrhs * (m + 1), 0.0), cs(nrhs * m),
        sn(nrhs * m);
    for (int c = 0; c < nrhs; c++) g[c * (m + 1)] = rn[c];
    int jdone = 0;
    for (int j = 0; j < m; j++) {
      do_sweeps(F, pV + j * nn, pZ + j * nn, nrhs, true, false);
      apply_A(F, pZ + j * nn, pw, nrhs, std::is_same<T, float>::value);
      std::vector<double> hh, hh2, hn;
      dots(pV, j + 1, pw, hh);  // hh[c * (j+1) + i]
      std::vector<double> neg(hh.size());
      for (size_t q = 0; q < hh.size(); q++) neg[q] = -hh[q];
      comb(pw, 1.0, pV, j + 1, neg);
      dots(pV, j + 1, pw, hh2);
      for (size_t q = 0; q < hh2.size(); q++) neg[q] = -hh2[q], hh[q] += hh2[q];
      comb(pw, 1.0, pV, j + 1, neg);
      dots(pw, 1, pw, hn);
      std::vector<double> invn(nrhs);
      double worst = 0;
      for (int c = 0; c < nrhs; c++) {
        double hnc = sqrt(std::max(hn[c], 0.0));
        invn[c] = hnc > 0 ? 1.0 / hnc : 0.0;
        double *Hc = &H[(size_t)c * (m + 1) * m];
        for (int i = 0; i <= j; i++) Hc[i * m + j] = hh[c * (j + 1) + i];
        Hc[(j + 1) * m + j] = hnc;
        // previous rotations, then a new one zeroing H[j+1][j]
        for (int i = 0; i < j; i++) {
          double a0 = Hc[i * m + j], a1 = Hc[(i + 1) * m + j];
          Hc[i * m + j] = cs[c * m + i] * a0 + sn[c * m + i] * a1;
          Hc[(i + 1) * m + j] = -sn[c * m + i] * a0 + cs[c * m + i] * a1;
        }
        double a0 = Hc[j * m + j], a1 = Hc[(j + 1) * m + j];
        double rr = hypot(a0, a1);
        double cc = rr > 0 ? a0 / rr : 1.0, ss = rr > 0 ? a1 / rr : 0.0;
        cs[c * m + j] = cc;
        sn[c * m + j] = ss;
        Hc[j * m + j] = rr;
        Hc[(j + 1) * m + j] = 0.0;
        double *gc = &g[(size_t)c * (m + 1)];
        gc[j + 1] = -ss * gc[j];
        gc[j] = cc * gc[j];
        worst = std::max(worst, fabs(gc[j + 1]) / bn[c]);
      }
      CK(cudaMemsetAsync(pV + (j + 1) * nn, 0, sizeof(double) * nn, st));
      comb(pV + (j + 1) * nn, 0.0, pw, 1, invn);
      inner++;
      jdone = j + 1;
      if (worst <= 0.5 * tol) break;
    }
    // y = H^{-1} g (upper triangular), x += Z y
    std::vector<double> y((size_t)nrhs * jdone);
    for (int c = 0; c < nrhs; c++) {
      const double *Hc = &H[(size_t)c * (m + 1) * m];
      const double *gc = &g[(size_t)c * (m + 1)];
      for (int i = jdone - 1; i >= 0; i--) {
        double sacc = gc[i];
        for (int l = i + 1; l < jdone; l++) sacc -= Hc[i * m + l] * y[c * jdone + l];
        y[c * jdone + i] = Hc[i * m + i] != 0 ? sacc / Hc[i * m + i] : 0.0;
      }
    }
    comb(x, 1.0, pZ, jdone, y);
  }
  if (iters) *iters = inner;
  if (relres) *relres = rel;
  CK(cudaStreamSynchronize(st));
  prof_collect(F);
  return ok;
}

// Conjugate gradients on A x = b preconditioned by the factor (the paper's
// solver for its examples, Sec. 4: F is symmetric for symmetric kernels,
// V_i = W_i^T).  FP64 vectors and residual operator; the preconditioner is
// the factor's solve (FP32 for the mixed factor, whose rounding makes it not
// quite symmetric, hence the flexible (Polak-Ribiere) form of beta).  All
// right-hand sides advance in lock step; a column whose residual is met, or
// whose curvature p^T A p is not positive, stops moving.  The recurrence
// residual decides when to stop; the true residual b - A x is then checked,
// and CG restarts from x if it is not met (within maxit iterations in all).
template <typename T>
static bool pcg(const Factor<T> &F, const double *b, double *x, int nrhs, double tol, int maxit, int *iters,
                double *relres) {
  cudaStream_t st = F.st;
  const int64_t n = F.n, nn = n * nrhs;
  DBuf R2, Z, P, Q, part, dres;
  R2.alloc(sizeof(double) * nn * 2, st);
  Z.alloc(sizeof(double) * nn, st);
  P.alloc(sizeof(double) * nn, st);
  Q.alloc(sizeof(double) * nn, st);
  part.alloc(sizeof(double) * 2 * nrhs * 240, st);
  dres.alloc(sizeof(double) * 2 * nrhs * 2, st);
  double *r = ptr<double>(R2), *rold = r + nn, *z = ptr<double>(Z), *p = ptr<double>(P), *q = ptr<double>(Q);
  double *dd = ptr<double>(dres), *dc = dd + 2 * nrhs;
  auto dots = [&](const double *Vb, int nv, const double *vec, std::vector<double> &out) {
    multidot(Vb, nn, nv, vec, n, nrhs, ptr<double>(part), dd, st);
    check_launch("multidot");
    out.resize((size_t)nv * nrhs);
    CK(cudaMemcpyAsync(out.data(), dd, sizeof(double) * nv * nrhs, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  };
  auto comb = [&](double *y, double alpha, const double *Vb, const std::vector<double> &coef) {
    staged_h2d(dc, coef.data(), sizeof(double) * nrhs, st);
    combine(y, alpha, Vb, nn, 1, dc, n, nrhs, st);
    check_launch("combine");
  };
  auto copy = [&](double *dst, const double *src) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
  };
  std::vector<double> bn, tmp;
  dots(b, 1, b, bn);
  for (auto &v : bn) v = v > 0 ? sqrt(v) : 1.0;
  // x0 = F^{-1} b
  do_sweeps(F, b, x, nrhs, true, false);
  int inner = 0;
  double rel = 0;
  bool ok = false;
  while (true) {
    // true residual r = b - A x
    apply_A(F, x, q, nrhs);
    copy(r, b);
    comb(r, 1.0, q, std::vector<double>(nrhs, -1.0));
    dots(r, 1, r, tmp);
    rel = 0;
    for (int c = 0; c < nrhs; c++) rel = std::max(rel, sqrt(std::max(tmp[c], 0.0)) / bn[c]);
    if (rel <= tol) {
      ok = true;
      break;
    }
    if (inner >= maxit) break;
    std::vector<char> live(nrhs);
    for (int c = 0; c < nrhs; c++) live[c] = sqrt(std::max(tmp[c], 0.0)) / bn[c] > tol;
    do_sweeps(F, r, z, nrhs, true, false);  // z = F^{-1} r
    copy(p, z);
    std::vector<double> rz;
    dots(r, 1, z, rz);
    while (inner < maxit) {
      apply_A(F, p, q, nrhs);  // q = A p
      std::vector<double> pq, alpha(nrhs, 0.0);
      dots(p, 1, q, pq);
      for (int c = 0; c < nrhs; c++) {
        if (live[c] && pq[c] > 0 && rz[c] > 0) alpha[c] = rz[c] / pq[c];
        else live[c] = 0;
      }
      comb(x, 1.0, p, alpha);
      copy(rold, r);
      for (auto &a : alpha) a = -a;
      comb(r, 1.0, q, alpha);
      inner++;
      dots(r, 1, r, tmp);
      double rr = 0;
      for (int c = 0; c < nrhs; c++) {
        const double rc = sqrt(std::max(tmp[c], 0.0)) / bn[c];
        if (rc <= tol) live[c] = 0;
        rr = std::max(rr, rc);
      }
      if (rr <= tol) break;
      do_sweeps(F, r, z, nrhs, true, false);
      std::vector<double> zr, beta(nrhs, 0.0);
      dots(r, 2, z, zr);  // zr[2c] = r.z, zr[2c+1] = r_old.z
      for (int c = 0; c < nrhs; c++) {
        if (live[c] && rz[c] > 0) beta[c] = (zr[2 * c] - zr[2 * c + 1]) / rz[c];
        rz[c] = zr[2 * c];
      }
      // p = z + beta p (q is free until the next product)
      copy(q, z);
      comb(q, 1.0, p, beta);
      std::swap(p, q);
    }
  }
  if (iters) *iters = inner;
  if (relres) *relres = rel;
  CK(cudaStreamSynchronize(st));
  prof_collect(F);
  return ok;
}

// Columns per pass of the sweep kernels: few enough for their shared-memory
// vectors (3 b x columns entries of the widest box within 200 KB).
template <typename T> static int sweep_columns(const Factor<T> &F, int nrhs) {
  int bm = 1;
  for (const auto &p : F.phases) bm = std::max(bm, p.bmax);
  return (int)std::max<size_t>(1, std::min<size_t>(nrhs, (size_t)(200 << 10) / ((size_t)3 * bm * sizeof(T))));
}

// Generalized square root (the remark after Eq. 3.11): for symmetric
// positive definite A the factor is F = V D W with W = V^T, so with
// D = C C^T (C block lower triangular, the Cholesky factors of the X_RR
// blocks and of the top blocks) F^{1/2} = V C satisfies
// F = F^{1/2} (F^{1/2})^T.  y = V C x applies C on every block's DOFs, then
// the apply's backward sweeps (the V product); (F^{1/2})^T x = C^T W x runs
// the apply's forward sweeps without D (the W product), then C^T.  The
// factors C are rebuilt once from the stored LU factors (X = P^T L U, then
// the Cholesky factor of its symmetric part).
template <typename T> static void chol_prepare(const Factor<T> &F) {
  if (F.chol_ready) return;
  cudaStream_t st = F.st;
  const int nbox = (int)F.h_boxes.size(), np = F.nprob;
  std::vector<int64_t> coff(nbox + np + 1, 0);
  int rmax = 1;
  for (int q = 0; q < nbox; q++) {
    const int r = F.h_boxes[q].r;
    coff[q + 1] = coff[q] + (int64_t)r * r;
    rmax = std::max(rmax, r);
  }
  for (int p = 0; p < np; p++) {
    const int t = F.ntop > 0 ? F.h_tn[p] : 0;
    if (t > 4096) throw Fail{RSS_EINVAL, "rss_sqrt_apply: top block larger than 4096"};
    coff[nbox + p + 1] = coff[nbox + p] + (int64_t)t * t;
    rmax = std::max(rmax, t);
  }
  upload(F.d_coff, coff, st);
  F.d_chol.alloc(sizeof(T) * std::max<int64_t>(coff.back(), 1), st);
  F.d_cerr.alloc(sizeof(int), st);
  CK(cudaMemsetAsync(F.d_cerr.p, 0, sizeof(int), st));
  launch_chol_from_lu<T>(ptr<FBox<T>>(F.d_boxes), nbox, F.ntop > 0 ? ptr<T>(F.d_topLU) : nullptr,
                         ptr<int64_t>(F.d_loff), ptr<int>(F.d_toppiv), ptr<int64_t>(F.d_toff), ptr<int>(F.d_tn),
                         F.ntop > 0 ? np : 0, ptr<T>(F.d_chol), ptr<int64_t>(F.d_coff), ptr<int>(F.d_cerr), st);
  check_launch("cholesky factors");
  int e = 0;
  CK(cudaMemcpyAsync(&e, F.d_cerr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (e) throw Fail{RSS_ENUMERIC, "rss_sqrt_apply: a diagonal block of D is not positive definite"};
  F.chol_rmax = rmax;
  F.chol_ready = true;
}

template <typename T>
static void sqrt_apply(const Factor<T> &F, const double *x, double *y, int nrhs, int trans) {
  chol_prepare(F);
  cudaStream_t st = F.st;
  const int nbox = (int)F.h_boxes.size(), np = F.ntop > 0 ? F.nprob : 0;
  // columns per pass: the sweeps' limit, and the block vectors within 200 KB
  int c = sweep_columns(F, nrhs);
  while (c > 1 && (size_t)F.chol_rmax * c * sizeof(T) > (size_t)(200 << 10)) c--;
  ensure_work(F, c);
  T *v = ptr<T>(F.d_work);
  for (int c0 = 0; c0 < nrhs; c0 += c) {
    const int nc = std::min(c, nrhs - c0);
    launch_permute<T>(0, ptr<int64_t>(F.d_perm), x + (size_t)c0 * F.n, v, nullptr, F.n, nc, st);
    auto blocks = [&](int tr) {
      launch_chol_apply<T>(ptr<FBox<T>>(F.d_boxes), nbox, ptr<int64_t>(F.d_top), ptr<int64_t>(F.d_toff),
                           ptr<int>(F.d_tn), np, ptr<T>(F.d_chol), ptr<int64_t>(F.d_coff), v, nc, F.chol_rmax, tr,
                           st);
    };
    if (!trans) {
      blocks(0);
      for (auto it = F.phases.rbegin(); it != F.phases.rend(); ++it) sweep_phase<T>(F, SWEEP_APPLY_BWD, *it, v, nc, st);
    } else {
      for (const Phase &p : F.phases) sweep_phase<T>(F, SWEEP_APPLY_W, p, v, nc, st);
      blocks(1);
    }
    launch_permute<T>(1, ptr<int64_t>(F.d_perm), nullptr, v, y + (size_t)c0 * F.n, F.n, nc, st);
    check_launch("rss_sqrt_apply");
  }
  if (!F.async()) CK(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------------------
// Allocation-free solve.  Its working vectors live in one fixed file-scope
// device array instead of memory allocated per factor: every device that
// loads this library holds the array until the process exits, every call
// shares it, and calls whose work overlaps on the GPU would race on it.
// ---------------------------------------------------------------------------

static constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[256];

// Device address of the scratch array for the current device, looked up on
// the first call made with that device current.  The same first call raises
// the sweep kernels' shared-memory limits on that device, so that no later
// call has to (a later call may be running under stream capture).
static void *noalloc_scratch() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) throw Fail{RSS_ECUDA, "rss_solve_noalloc: device ordinal out of range"};
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Fail{RSS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
    }
    sweep_kernel_attributes();
    e = cudaGetLastError();
    if (e != cudaSuccess) throw Fail{RSS_ECUDA, std::string("sweep kernel attributes: ") + cudaGetErrorString(e)};
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}


// The solve of Eq. 3.11 in passes of at most `c` columns, each pass with its
// n x c working vector and 2 x ntop x c top-block entries in the fixed array.
template <typename T>
static void solve_noalloc(const Factor<T> &F, const double *b, double *x, int nrhs) {
  auto vbytes = [&](int c) { return (((size_t)F.n * c * sizeof(T)) + 255) & ~(size_t)255; };
  auto tbytes = [&](int c) { return (size_t)2 * F.ntop * c * sizeof(T); };
  int c = sweep_columns(F, nrhs);
  while (c > 0 && vbytes(c) + tbytes(c) > NOALLOC_SCRATCH_BYTES) c--;
  if (c < 1) throw Fail{RSS_EINVAL, "rss_solve_noalloc: one column of n entries exceeds the fixed 16 MiB scratch"};
  unsigned char *base = static_cast<unsigned char *>(noalloc_scratch());
  T *v = reinterpret_cast<T *>(base);
  T *topwork = reinterpret_cast<T *>(base + vbytes(c));
  cudaStream_t st = F.st;
  for (int c0 = 0; c0 < nrhs; c0 += c) {
    const int nc = std::min(c, nrhs - c0);
    const double *bc = b + (size_t)c0 * F.n;
    double *xc = x + (size_t)c0 * F.n;
    launch_permute<T>(0, ptr<int64_t>(F.d_perm), bc, v, nullptr, F.n, nc, st);
    for (const Phase &p : F.phases) sweep_phase<T>(F, SWEEP_SOLVE_FWD, p, v, nc, st);
    launch_top<T>(0, ptr<T>(F.d_topLU), ptr<int64_t>(F.d_loff), ptr<int>(F.d_toppiv), ptr<int64_t>(F.d_top),
                  ptr<int64_t>(F.d_toff), ptr<int>(F.d_tn), F.nprob, F.ntop, v, nc, topwork, st,
                  F.d_topinv.p ? ptr<T>(F.d_topinv) : nullptr);
    for (auto it = F.phases.rbegin(); it != F.phases.rend(); ++it) sweep_phase<T>(F, SWEEP_SOLVE_BWD, *it, v, nc, st);
    launch_permute<T>(1, ptr<int64_t>(F.d_perm), nullptr, v, xc, F.n, nc, st);
    check_launch("rss_solve_noalloc");
  }
  if (!F.async()) CK(cudaStreamSynchronize(st));
}

// Columns in chunks small enough for the sweep kernels' shared-memory
// vectors (3 b x columns entries of the widest box within 200 KB); calls of
// up to 4 columns on factors of boxes up to ~2000 wide are one chunk.
template <typename T> static void sweeps_chunked(const Factor<T> &F, const double *in, double *out, int nrhs,
                                                 bool solve) {
  const int cmax = sweep_columns(F, nrhs);
  for (int c0 = 0; c0 < nrhs; c0 += cmax)
    do_sweeps(F, in + (size_t)c0 * F.n, out + (size_t)c0 * F.n, std::min(cmax, nrhs - c0), solve);
}

static rss_status sweep_entry(const rss_factorization *f, const double *in, double *out, int nrhs, bool solve) {
  return guard([&] {
    if (!f || !f->impl || nrhs < 1) throw Fail{RSS_EINVAL, "bad arguments"};
    if (f->impl->prec == RSS_FP64) {
      auto &F = static_cast<const Factor<double> &>(*f->impl);
      take_deferred(F, false);
      if (F.n > 0 && (!in || !out)) throw Fail{RSS_EINVAL, "NULL vector"};
      sweeps_chunked(F, in, out, nrhs, solve);
    } else {
      auto &F = static_cast<const Factor<float> &>(*f->impl);
      take_deferred(F, false);
      if (F.n > 0 && (!in || !out)) throw Fail{RSS_EINVAL, "NULL vector"};
      sweeps_chunked(F, in, out, nrhs, solve);
    }
  });
}

// Every other entry point on a factor reads a deferred device error first.
static void take_deferred_any(const rss_factorization *f, bool wait) {
  if (f->impl->prec == RSS_FP64) take_deferred(static_cast<const Factor<double> &>(*f->impl), wait);
  else take_deferred(static_cast<const Factor<float> &>(*f->impl), wait);
}

extern "C" {

const char *rss_last_error(void) { return g_last_error.c_str(); }

int64_t rss_kernel_launches(void) { return (int64_t)launches_total(); }

rss_status rss_build_tree(const double *pts, int64_t n, int dim, int leaf_size, rss_tree **out) {
  return guard([&] {
    if (!out || n < 0 || (dim != 2 && dim != 3) || leaf_size < 1 || (n > 0 && !pts))
      throw Fail{RSS_EINVAL, "rss_build_tree: bad arguments"};
    std::unique_ptr<rss_tree> tr(new rss_tree());
    std::vector<HTree> one(1);
    const double *pp[1] = {pts};
    build_trees_gpu(one, pp, &n, 1, dim, leaf_size, nullptr);
    tr->t = std::move(one[0]);
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

// Factor one or several independent problems into one handle.
static rss_status factor_impl(int nprob, const double *const *pts, const int64_t *n, int dim, rss_kernel kernel,
                              double eps, int leaf_size, const rss_options *opts, rss_factorization **out) {
  return guard([&] {
    if (!out || nprob < 1 || !pts || !n || (dim != 2 && dim != 3) || leaf_size < 1 || !(eps >= 0.0) ||
        (kernel.kind != RSS_LAPLACE2D_LOG && kernel.kind != RSS_LAPLACE3D_INV))
      throw Fail{RSS_EINVAL, "rss_factor: bad arguments"};
    for (int p = 0; p < nprob; p++)
      if (n[p] < 0 || (n[p] > 0 && !pts[p])) throw Fail{RSS_EINVAL, "rss_factor: bad arguments"};
    rss_options o{};
    if (opts) o = *opts;
    const bool prof_on = o.profile != 0;
    if (o.prec != RSS_FP64 && o.prec != RSS_MIXED) throw Fail{RSS_EINVAL, "rss_factor: bad precision"};
    if ((o.flags & RSS_FLAG_HYBRID) && ((o.flags & RSS_FLAG_COLOUR_2D) || o.mlp))
      throw Fail{RSS_EINVAL, "rss_factor: the hybrid factorization takes neither the 2^d schedule nor a rank proposal"};
    cudaStream_t st = (cudaStream_t)o.stream;
    const MlpModel *mlp = nullptr;
    if (o.mlp) {
      if (o.mlp->magic != MAGIC_MLP || !o.mlp->impl) throw Fail{RSS_EINVAL, "rss_factor: bad rank-proposal handle"};
      mlp = o.mlp->impl.get();
    }
    std::unique_ptr<rss_factorization> res(new rss_factorization());
    auto setup = [&](auto *F) {
      F->st = st;
      F->dim = dim;
      F->nprob = nprob;
      F->trees.resize(nprob);
      F->pdof.assign(nprob + 1, 0);
      F->pw.assign(nprob, 1.0);
      for (int p = 0; p < nprob; p++) {
        F->pdof[p + 1] = F->pdof[p] + n[p];
        F->pw[p] = kernel.weight > 0 ? kernel.weight : (n[p] > 0 ? 1.0 / (double)n[p] : 1.0);
        F->trees[p].dim = dim;
        F->trees[p].leaf = leaf_size;
        F->trees[p].n = n[p];
      }
      F->n = F->pdof[nprob];
      // the trees of every problem, built on the GPU in one pass
      double tt0 = now_ms();
      build_trees_gpu(F->trees, pts, n, nprob, dim, leaf_size, st, &F->dev_pts);
      F->prof.host(KC_HOST_TREE, now_ms() - tt0);
      F->K.kind = kernel.kind;
      F->K.diag = kernel.diag;
      F->K.w = F->pw[0];
      F->px.np = o.n_proxy > 0 ? o.n_proxy : (dim == 2 ? 64 : 512);
      F->px.radius = o.proxy_radius > 0 ? o.proxy_radius : 2.5;
      F->eps = eps;
      F->flags = o.flags;
      F->use_graphs = o.use_graphs != 0;
      run_factor(*F);
    };
    // A proposal that leaves a level short of storage costs one more run with
    // full-size reservations; the ranks (and so the factor) are the same.
    for (int attempt = 0;; attempt++) {
      try {
        if (o.prec == RSS_FP64) {
          auto *F = new Factor<double>();
          res->impl.reset(F);
          F->prec = RSS_FP64;
          F->prof.on = prof_on;
          F->mlp = attempt == 0 ? mlp : nullptr;
          F->retries = attempt;
          setup(F);
        } else {
          auto *F = new Factor<float>();
          res->impl.reset(F);
          F->prec = RSS_MIXED;
          F->prof.on = prof_on;
          F->mlp = attempt == 0 ? mlp : nullptr;
          F->retries = attempt;
          setup(F);
        }
        break;
      } catch (const Retry &) {
        if (attempt > 0) throw Fail{RSS_ECUDA, "storage check failed with full-size reservations"};
        CK(cudaStreamSynchronize(st));
      }
    }
    *out = res.release();
  });
}

rss_status rss_factor(const double *pts, int64_t n, int dim, rss_kernel kernel, double eps, int leaf_size,
                      const rss_options *opts, rss_factorization **out) {
  const double *p[1] = {pts};
  int64_t nn[1] = {n};
  return factor_impl(1, p, nn, dim, kernel, eps, leaf_size, opts, out);
}

rss_status rss_factor_batched(int nprob, const double *const *pts, const int64_t *n, int dim, rss_kernel kernel,
                              double eps, int leaf_size, const rss_options *opts, rss_factorization **out) {
  return factor_impl(nprob, pts, n, dim, kernel, eps, leaf_size, opts, out);
}

rss_status rss_solve_refined(const rss_factorization *f, const double *b, double *x, int nrhs, double tol,
                             int maxit, int *iters, double *relres) {
  bool ok = false;
  rss_status stt = guard([&] {
    if (!f || !f->impl || nrhs < 1 || !(tol > 0) || maxit < 0) throw Fail{RSS_EINVAL, "rss_solve_refined: bad arguments"};
    take_deferred_any(f, true);
    if (f->impl->prec == RSS_FP64) {
      auto &F = static_cast<const Factor<double> &>(*f->impl);
      if (F.n > 0 && (!b || !x)) throw Fail{RSS_EINVAL, "NULL vector"};
      ok = F.n == 0 || refine(F, b, x, nrhs, tol, maxit, iters, relres);
    } else {
      auto &F = static_cast<const Factor<float> &>(*f->impl);
      if (F.n > 0 && (!b || !x)) throw Fail{RSS_EINVAL, "NULL vector"};
      ok = F.n == 0 || refine(F, b, x, nrhs, tol, maxit, iters, relres);
    }
  });
  if (stt == RSS_OK && !ok) {
    g_last_error = "rss_solve_refined: tolerance not reached";
    return RSS_ENOTCONV;
  }
  return stt;
}

rss_status rss_solve_cg(const rss_factorization *f, const double *b, double *x, int nrhs, double tol, int maxit,
                        int *iters, double *relres) {
  bool ok = false;
  rss_status stt = guard([&] {
    if (!f || !f->impl || nrhs < 1 || !(tol > 0) || maxit < 0) throw Fail{RSS_EINVAL, "rss_solve_cg: bad arguments"};
    take_deferred_any(f, true);
    auto run = [&](const auto &F) {
      if (F.n > 0 && (!b || !x)) throw Fail{RSS_EINVAL, "NULL vector"};
      ok = F.n == 0 || pcg(F, b, x, nrhs, tol, maxit, iters, relres);
    };
    if (f->impl->prec == RSS_FP64) run(static_cast<const Factor<double> &>(*f->impl));
    else run(static_cast<const Factor<float> &>(*f->impl));
  });
  if (stt == RSS_OK && !ok) {
    g_last_error = "rss_solve_cg: tolerance not reached";
    return RSS_ENOTCONV;
  }
  return stt;
}

rss_status rss_apply(const rss_factorization *f, const double *x, double *y, int nrhs) {
  return sweep_entry(f, x, y, nrhs, false);
}

rss_status rss_solve(const rss_factorization *f, const double *b, double *x, int nrhs) {
  return sweep_entry(f, b, x, nrhs, true);
}

rss_status rss_solve_noalloc(const rss_factorization *f, const double *b, double *x, int nrhs) {
  return guard([&] {
    if (!f || !f->impl || nrhs < 1) throw Fail{RSS_EINVAL, "rss_solve_noalloc: bad arguments"};
    take_deferred_any(f, false);
    if (f->impl->prec == RSS_FP64) {
      auto &F = static_cast<const Factor<double> &>(*f->impl);
      if (F.n > 0 && (!b || !x)) throw Fail{RSS_EINVAL, "NULL vector"};
      solve_noalloc(F, b, x, nrhs);
    } else {
      auto &F = static_cast<const Factor<float> &>(*f->impl);
      if (F.n > 0 && (!b || !x)) throw Fail{RSS_EINVAL, "NULL vector"};
      solve_noalloc(F, b, x, nrhs);
    }
  });
}

rss_status rss_sqrt_apply(const rss_factorization *f, const double *x, double *y, int nrhs, int transpose) {
  return guard([&] {
    if (!f || !f->impl || nrhs < 1 || (transpose != 0 && transpose != 1))
      throw Fail{RSS_EINVAL, "rss_sqrt_apply: bad arguments"};
    take_deferred_any(f, false);
    auto run = [&](const auto &F) {
      if (F.n > 0 && (!x || !y)) throw Fail{RSS_EINVAL, "NULL vector"};
      if (F.n > 0) sqrt_apply(F, x, y, nrhs, transpose);
    };
    if (f->impl->prec == RSS_FP64) run(static_cast<const Factor<double> &>(*f->impl));
    else run(static_cast<const Factor<float> &>(*f->impl));
  });
}

rss_status rss_matvec(const rss_factorization *f, const double *x, double *y, int nrhs) {
  return guard([&] {
    if (!f || !f->impl || nrhs < 1) throw Fail{RSS_EINVAL, "rss_matvec: bad arguments"};
    take_deferred_any(f, false);
    auto run = [&](const auto &F) {
      if (F.n > 0 && (!x || !y)) throw Fail{RSS_EINVAL, "NULL vector"};
      if (F.n > 0) apply_A(F, x, y, nrhs);
      if (!F.async()) CK(cudaStreamSynchronize(F.st));
    };
    if (f->impl->prec == RSS_FP64) run(static_cast<const Factor<double> &>(*f->impl));
    else run(static_cast<const Factor<float> &>(*f->impl));
  });
}

rss_status rss_sync(const rss_factorization *f) {
  return guard([&] {
    if (!f || !f->impl) throw Fail{RSS_EINVAL, "rss_sync: bad arguments"};
    auto run = [&](const auto &F) {
      CK(cudaStreamSynchronize(F.st));
      take_deferred(F, true);
    };
    if (f->impl->prec == RSS_FP64) run(static_cast<const Factor<double> &>(*f->impl));
    else run(static_cast<const Factor<float> &>(*f->impl));
  });
}

rss_status rss_logdet(const rss_factorization *f, double *logabs) {
  return guard([&] {
    if (!f || !f->impl || !logabs) throw Fail{RSS_EINVAL, "rss_logdet: bad arguments"};
    take_deferred_any(f, true);
    auto run = [&](const auto &F) {
      using T = typename std::remove_reference_t<decltype(F)>::value_type;
      const int nbox = (int)F.h_boxes.size(), np = F.nprob;
      DBuf part, first;
      part.alloc(sizeof(double) * ((size_t)nbox + np) + 16, F.st);
      first.alloc(sizeof(int64_t) * (size_t)nbox + 16, F.st);
      launch_logdet<T>(ptr<FBox<T>>(F.d_boxes), nbox, F.ntop > 0 ? ptr<T>(F.d_topLU) : nullptr,
                       ptr<int64_t>(F.d_loff), ptr<int>(F.d_tn), F.ntop > 0 ? np : 0, ptr<double>(part),
                       ptr<int64_t>(first), F.st);
      check_launch("logdet");
      std::vector<double> hp((size_t)nbox + np, 0.0);
      std::vector<int64_t> hf(nbox);
      if (nbox > 0)
        CK(cudaMemcpyAsync(hf.data(), first.p, sizeof(int64_t) * nbox, cudaMemcpyDeviceToHost, F.st));
      CK(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * (nbox + (F.ntop > 0 ? np : 0)),
                         cudaMemcpyDeviceToHost, F.st));
      CK(cudaStreamSynchronize(F.st));
      // boxes in factor order, then the top block, per problem
      for (int p = 0; p < np; p++) logabs[p] = 0.0;
      for (int q = 0; q < nbox; q++) {
        if (hf[q] < 0) continue;
        const int p = (int)(std::upper_bound(F.pdof.begin(), F.pdof.end(), hf[q]) - F.pdof.begin()) - 1;
        if (p >= 0 && p < np) logabs[p] += hp[q];
      }
      if (F.ntop > 0)
        for (int p = 0; p < np; p++) logabs[p] += hp[(size_t)nbox + p];
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
      const int64_t sz = F.prec == RSS_FP64 ? 8 : 4;
      s = {(int64_t)F.h_boxes.size(), F.ntop, F.factor_bytes, F.maxdepth, F.n, F.prec, F.reserved_T * sz,
           F.used_T * sz, F.ovf_used * sz, F.retries, F.mlp ? 1 : 0};
      for (const auto &b : F.h_boxes) {
        s.push_back(b.depth);
        s.push_back(b.b);
        s.push_back(b.k);
        s.push_back(b.nj);
        s.push_back(b.rres);
        s.push_back(b.njres);
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

rss_status rss_stats_json(const rss_factorization *f, char *buf, size_t *nbytes) {
  return guard([&] {
    if (!f || !f->impl || !nbytes) throw Fail{RSS_EINVAL, "rss_stats_json: bad arguments"};
    std::string js;
    auto num = [&](const char *key, double v, bool comma = true) {
      char tmp[96];
      snprintf(tmp, sizeof(tmp), "\"%s\": %.17g%s", key, v, comma ? ", " : "");
      js += tmp;
    };
    auto fill = [&](const auto &F) {
      const int64_t sz = F.prec == RSS_FP64 ? 8 : 4;
      js += "{";
      num("n", (double)F.n);
      num("problems", F.nprob);
      num("dim", F.dim);
      js += std::string("\"precision\": \"") + (F.prec == RSS_FP64 ? "fp64" : "fp32") + "\", ";
      num("eps", F.eps);
      num("colours_per_level", (F.flags & RSS_FLAG_COLOUR_2D) ? (1 << F.dim) : (F.dim == 2 ? 9 : 27));
      num("maxdepth", F.maxdepth);
      num("boxes", (double)F.h_boxes.size());
      num("top_block", F.ntop);
      num("factor_bytes", (double)F.factor_bytes);
      num("reserved_bytes", (double)(F.reserved_T * sz));
      num("used_bytes", (double)(F.used_T * sz));
      num("overflow_bytes", (double)(F.ovf_used * sz));
      num("retried", F.retries);
      num("rank_proposal", F.mlp ? 1 : 0);
      // per depth: boxes, sum and largest of |B|, k, |J|
      js += "\"levels\": [";
      bool first = true;
      for (int t = F.maxdepth; t >= 0; t--) {
        int64_t cnt = 0, sb = 0, sk = 0, sj = 0, mb = 0, mk = 0, mj = 0;
        for (const auto &b : F.h_boxes) {
          if (b.depth != t) continue;
          cnt++;
          sb += b.b, sk += b.k, sj += b.nj;
          mb = std::max<int64_t>(mb, b.b), mk = std::max<int64_t>(mk, b.k), mj = std::max<int64_t>(mj, b.nj);
        }
        if (!cnt) continue;
        js += first ? "{" : ", {";
        first = false;
        num("depth", t);
        num("boxes", (double)cnt);
        num("b_sum", (double)sb);
        num("k_sum", (double)sk);
        num("nj_sum", (double)sj);
        num("b_max", (double)mb);
        num("k_max", (double)mk);
        num("nj_max", (double)mj, false);
        js += "}";
      }
      js += "], ";
      // per box in elimination order: depth, |B|, k, |J|
      const char *names[4] = {"box_depth", "box_b", "box_k", "box_nj"};
      for (int q = 0; q < 4; q++) {
        js += std::string("\"") + names[q] + "\": [";
        for (size_t i = 0; i < F.h_boxes.size(); i++) {
          const auto &b = F.h_boxes[i];
          const int v = q == 0 ? b.depth : q == 1 ? b.b : q == 2 ? b.k : b.nj;
          js += (i ? ", " : "") + std::to_string(v);
        }
        js += "], ";
      }
      // kernel-class times when the factor was created with profiling
      const Prof &P = F.prof;
      static const char *cls[KC_N] = {"assemble", "id", "elim", "schur", "top_lu", "sweep", "top_solve",
                                      "permute", "host_tree", "host_level", "host_wait", "residual_operator",
                                      "inner_operator"};
      js += "\"profile_ms\": {";
      for (int c = 0; c < KC_N; c++) num(cls[c], P.ms[c], c + 1 < KC_N);
      js += "}}";
    };
    if (f->impl->prec == RSS_FP64) fill(static_cast<const Factor<double> &>(*f->impl));
    else fill(static_cast<const Factor<float> &>(*f->impl));
    const size_t need = js.size() + 1, cap = *nbytes;
    *nbytes = need;
    if (buf) {
      if (cap < need) throw Fail{RSS_EINVAL, "rss_stats_json: buffer too small"};
      memcpy(buf, js.c_str(), need);
    }
  });
}

rss_status rss_profile(const rss_factorization *f, int reset, double *buf, size_t *nbytes) {
  return guard([&] {
    if (!f || !f->impl || !nbytes) throw Fail{RSS_EINVAL, "rss_profile: bad arguments"};
    Prof &P = f->impl->prof;
    const size_t need = sizeof(double) * 4 * KC_N;
    size_t cap = *nbytes;
    *nbytes = need;
    if (buf) {
      if (cap < need) throw Fail{RSS_EINVAL, "rss_profile: buffer too small"};
      for (int c = 0; c < KC_N; c++) {
        buf[4 * c] = (double)P.launches[c];
        buf[4 * c + 1] = P.ms[c];
        buf[4 * c + 2] = P.bytes[c];
        buf[4 * c + 3] = P.flops[c];
      }
    }
    if (reset) P.reset();
  });
}

rss_status rss_box_features(const rss_factorization *f, float *feat, int32_t *rank, int64_t nbox) {
  return guard([&] {
    if (!f || !f->impl) throw Fail{RSS_EINVAL, "rss_box_features: bad arguments"};
    auto fill = [&](const auto &F) {
      if (nbox != (int64_t)F.h_boxes.size()) throw Fail{RSS_EINVAL, "rss_box_features: nbox does not match"};
      if (nbox > 0 && (!feat || !rank)) throw Fail{RSS_EINVAL, "rss_box_features: bad arguments"};
      if (nbox > 0) memcpy(feat, F.feats.data(), sizeof(float) * MLP_NFEAT * (size_t)nbox);
      for (int64_t q = 0; q < nbox; q++) rank[q] = F.h_boxes[q].k;
    };
    if (f->impl->prec == RSS_FP64) fill(static_cast<const Factor<double> &>(*f->impl));
    else fill(static_cast<const Factor<float> &>(*f->impl));
  });
}

// SplitMix64 (Steele, Lea and Flood 2014): output i of the stream seeded s is
// the finaliser applied to s + (i + 1) * 0x9E3779B97F4A7C15.
static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

rss_status rss_mlp_create(const float *params, uint64_t seed, void *stream, rss_mlp **out) {
  return guard([&] {
    if (!out) throw Fail{RSS_EINVAL, "rss_mlp_create: bad arguments"};
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<float> th(MLP_NPARAM, 0.f);
    if (params) {
      memcpy(th.data(), params, sizeof(float) * MLP_NPARAM);
    } else {
      // Glorot-uniform weights U(-s, s), s = sqrt(6 / (fan_in + fan_out)); zero biases
      const int H = MLP_HIDDEN, NF = MLP_NFEAT;
      struct Blk { int off, n, fin, fout; } blks[] = {
          {0, H * NF, NF, H}, {H * NF + H, H * H, H, H}, {H * NF + 2 * H + H * H, H * H, H, H},
          {H * NF + 3 * H + 2 * H * H, H, H, 1}};
      for (const Blk &b : blks) {
        const double sc = sqrt(6.0 / (b.fin + b.fout));
        for (int i = 0; i < b.n; i++) {
          const double u = (double)(splitmix64_at(seed, (uint64_t)(b.off + i)) >> 11) * 0x1.0p-53;
          th[b.off + i] = (float)((2.0 * u - 1.0) * sc);
        }
      }
    }
    std::unique_ptr<rss_mlp> h(new rss_mlp());
    h->impl.reset(new MlpModel());
    MlpModel &M = *h->impl;
    M.st = st;
    upload(M.theta, th, st);
    M.wbf.alloc(sizeof(uint16_t) * MLP_NPARAM, st);
    M.m.alloc(sizeof(float) * MLP_NPARAM, st);
    M.v.alloc(sizeof(float) * MLP_NPARAM, st);
    M.grad.alloc(sizeof(float) * MLP_NPARAM, st);
    M.step.alloc(sizeof(int), st);
    M.loss.alloc(sizeof(double), st);
    CK(cudaMemsetAsync(M.m.p, 0, sizeof(float) * MLP_NPARAM, st));
    CK(cudaMemsetAsync(M.v.p, 0, sizeof(float) * MLP_NPARAM, st));
    CK(cudaMemsetAsync(M.step.p, 0, sizeof(int), st));
    mlp_round(ptr<float>(M.theta), M.wbf.p, st);
    check_launch("mlp_round");
    CK(cudaStreamSynchronize(st));
    *out = h.release();
  });
}

static const MlpModel &mlp_of(const rss_mlp *m) {
  if (!m || m->magic != MAGIC_MLP || !m->impl) throw Fail{RSS_EINVAL, "bad rank-proposal handle"};
  return *m->impl;
}

rss_status rss_mlp_params(const rss_mlp *m, float *params) {
  return guard([&] {
    const MlpModel &M = mlp_of(m);
    if (!params) throw Fail{RSS_EINVAL, "rss_mlp_params: bad arguments"};
    CK(cudaMemcpyAsync(params, M.theta.p, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, M.st));
    CK(cudaStreamSynchronize(M.st));
  });
}

rss_status rss_mlp_predict(const rss_mlp *m, const float *X, int64_t n, float *y) {
  return guard([&] {
    const MlpModel &M = mlp_of(m);
    if (n < 0 || (n > 0 && (!X || !y))) throw Fail{RSS_EINVAL, "rss_mlp_predict: bad arguments"};
    mlp_forward(M.wbf.p, X, n, y, M.st);
    check_launch("mlp_forward");
    CK(cudaStreamSynchronize(M.st));
  });
}

rss_status rss_mlp_grad(const rss_mlp *m, const float *X, const float *y, int64_t n, float *grad, double *loss) {
  return guard([&] {
    const MlpModel &M = mlp_of(m);
    if (n < 1 || !X || !y || !grad) throw Fail{RSS_EINVAL, "rss_mlp_grad: bad arguments"};
    const int nblk = mlp_grad_blocks(n);
    DBuf part, lpart;
    part.alloc(sizeof(float) * (size_t)nblk * MLP_NPARAM, M.st);
    lpart.alloc(sizeof(double) * nblk, M.st);
    mlp_gradient(M.wbf.p, X, y, n, ptr<float>(part), ptr<double>(lpart), grad, ptr<double>(M.loss), M.st);
    check_launch("mlp_gradient");
    double l = 0;
    CK(cudaMemcpyAsync(&l, M.loss.p, sizeof(double), cudaMemcpyDeviceToHost, M.st));
    CK(cudaStreamSynchronize(M.st));
    if (loss) *loss = l;
  });
}

rss_status rss_mlp_train(rss_mlp *m, const float *X, const float *y, int64_t n, int iters, float lr, double *loss) {
  return guard([&] {
    MlpModel &M = const_cast<MlpModel &>(mlp_of(m));
    if (n < 1 || !X || !y || iters < 0 || !(lr > 0.f)) throw Fail{RSS_EINVAL, "rss_mlp_train: bad arguments"};
    const int nblk = mlp_grad_blocks(n);
    DBuf part, lpart;
    part.alloc(sizeof(float) * (size_t)nblk * MLP_NPARAM, M.st);
    lpart.alloc(sizeof(double) * nblk, M.st);
    if (iters > 0) {
      // one iteration (gradient, reduction, Adam) captured once, replayed
      cudaStream_t cs = nullptr;
      cudaEvent_t ev = nullptr;
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      auto cleanup = [&] {
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (ev) cudaEventDestroy(ev);
        if (cs) cudaStreamDestroy(cs);
      };
      try {
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, M.st));
        CK(cudaStreamWaitEvent(cs, ev, 0));
        // kernel attributes are set by an uncaptured gradient call first
        mlp_gradient(M.wbf.p, X, y, n, ptr<float>(part), ptr<double>(lpart), ptr<float>(M.grad),
                     ptr<double>(M.loss), cs);
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        mlp_gradient(M.wbf.p, X, y, n, ptr<float>(part), ptr<double>(lpart), ptr<float>(M.grad),
                     ptr<double>(M.loss), cs);
        mlp_adam(ptr<float>(M.theta), ptr<float>(M.m), ptr<float>(M.v), ptr<float>(M.grad), M.wbf.p,
                 ptr<int>(M.step), lr, cs);
        CK(cudaStreamEndCapture(cs, &g));
        count_launch(-3);  // the capture launched nothing
        CK(cudaGraphInstantiate(&ge, g, 0));
        for (int it = 0; it < iters; it++) CK(cudaGraphLaunch(ge, cs));
        count_launch(3 * iters);
        CK(cudaEventRecord(ev, cs));
        CK(cudaStreamWaitEvent(M.st, ev, 0));
      } catch (...) {
        if (cs) cudaStreamSynchronize(cs);
        cleanup();
        throw;
      }
      CK(cudaStreamSynchronize(M.st));
      cleanup();
    }
    double l = 0;
    CK(cudaMemcpyAsync(&l, M.loss.p, sizeof(double), cudaMemcpyDeviceToHost, M.st));
    CK(cudaStreamSynchronize(M.st));
    if (loss) *loss = l;
  });
}

rss_status rss_autotune_table(int32_t *buf, size_t *nbytes) {
  return guard([&] {
    if (!nbytes) throw Fail{RSS_EINVAL, "rss_autotune_table: bad arguments"};
    std::vector<int32_t> v;
    {
      std::lock_guard<std::mutex> lk(g_tune_m);
      for (const auto &kv : g_tune) {
        v.push_back(std::get<0>(kv.first));
        v.push_back(std::get<1>(kv.first));
        v.push_back(std::get<2>(kv.first));
        for (int f = 0; f < 4; f++) v.push_back(kTuneShapes[kv.second.shape][f]);
        for (int c = 0; c < kNShapes; c++) v.push_back((int32_t)std::lround(kv.second.us[c]));
      }
    }
    const size_t need = v.size() * sizeof(int32_t), cap = *nbytes;
    *nbytes = need;
    if (buf) {
      if (cap < need) throw Fail{RSS_EINVAL, "rss_autotune_table: buffer too small"};
      if (need) memcpy(buf, v.data(), need);
    }
  });
}

rss_status rss_autotune_set(int elem_bytes, int width, int phase_class, int tpc, int groups, int ctas, int rows) {
  return guard([&] {
    int shape = -1;
    for (int c = 0; c < kNShapes; c++)
      if (kTuneShapes[c][0] == tpc && kTuneShapes[c][1] == groups && kTuneShapes[c][2] == ctas &&
          kTuneShapes[c][3] == rows)
        shape = c;
    if (shape < 0 || (elem_bytes != 4 && elem_bytes != 8) || (width != 64 && width != 128 && width != 256) ||
        phase_class < 0 || phase_class > 40 || !shape_fits(width, tpc, groups, rows) ||
        (width == 256 && ctas > 1 && tpc != 2))
      throw Fail{RSS_EINVAL, "rss_autotune_set: bad arguments"};
    std::lock_guard<std::mutex> lk(g_tune_m);
    TuneEntry te{shape, {}};
    g_tune[std::make_tuple(elem_bytes, width, phase_class)] = te;
  });
}

rss_status rss_autotune_elim_table(int32_t *buf, size_t *nbytes) {
  return guard([&] {
    if (!nbytes) throw Fail{RSS_EINVAL, "rss_autotune_elim_table: bad arguments"};
    std::vector<int32_t> v;
    {
      std::lock_guard<std::mutex> lk(g_tune_m);
      for (const auto &kv : g_tune_elim) {
        v.push_back(std::get<0>(kv.first));
        v.push_back(std::get<1>(kv.first));
        v.push_back(std::get<2>(kv.first));
        for (int f = 0; f < 2; f++) v.push_back(kElimShapes[kv.second.shape][f]);
        for (int c = 0; c < kNElim; c++) v.push_back((int32_t)std::lround(kv.second.us[c]));
      }
    }
    const size_t need = v.size() * sizeof(int32_t), cap = *nbytes;
    *nbytes = need;
    if (buf) {
      if (cap < need) throw Fail{RSS_EINVAL, "rss_autotune_elim_table: buffer too small"};
      if (need) memcpy(buf, v.data(), need);
    }
  });
}

void rss_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_m);
  g_tune.clear();
  g_tune_elim.clear();
}

void rss_free(void *handle) {
  if (!handle) return;
  // every handle type starts with a distinct 32-bit tag
  uint32_t magic = *static_cast<const uint32_t *>(handle);
  if (magic == MAGIC_TREE) delete static_cast<rss_tree *>(handle);
  else if (magic == MAGIC_FACTOR) delete static_cast<rss_factorization *>(handle);
  else if (magic == MAGIC_MLP) delete static_cast<rss_mlp *>(handle);
}

}  // extern "C"
