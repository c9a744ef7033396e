// refine.cu -- FP64 residual operator and vector kernels of the iterative
// refinement (GMRES-IR) around the factorization.
//
// When the points are the cell centres of an s^d grid, K_ij = kappa(I_i - I_j)
// depends only on the integer offset of the two cells, so K x is a discrete
// convolution.  It is applied exactly (to FP64 rounding) by embedding the
// kernel in a circulant of side L = 2s and using a Stockham FFT written here
// (radix-4 passes, one CTA per line, the line held in shared memory).  Two real
// right-hand sides share one complex transform (x1 + i x2): the embedded
// kernel is real and even, so its spectrum is real and the real and
// imaginary parts of the product transform back to K x1 and K x2.
//
// This operator is the FP64 residual r = b - A x of the iterative
// refinement; it is not part of the factorization itself.  The same
// transforms in FP32 (spectrum and twiddles rounded from their FP64 values)
// are the operator products inside the refinement's inner GMRES for a FP32
// factor: there an operator accurate to FP32 rounding is enough (the inner
// solve only has to shrink the correction's error by a bounded factor), and
// FP64 stays for the residuals and the update.
#include <cuda_runtime.h>

#include "internal.h"

namespace rss {

// complex type of a real type, its constructor and fused multiply-add
template <typename R> struct Cx;
template <> struct Cx<double> {
  using t = double2;
  static __device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }
  static __device__ __forceinline__ double fm(double a, double b, double c) { return fma(a, b, c); }
};
template <> struct Cx<float> {
  using t = float2;
  static __device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
  static __device__ __forceinline__ float fm(float a, float b, float c) { return fmaf(a, b, c); }
};

// One Stockham FFT of length L (power of two, L <= 2048; radix 4, with one
// radix-2 pass when log2 L is odd) per CTA
// over lines of a complex array: line q starts at base(q) and has stride
// `stride`; lines are enumerated as q = q0 + blockIdx.x.  sign = -1 forward,
// +1 inverse (unscaled).
template <typename R>
__global__ void __launch_bounds__(256) k_fft_lines(typename Cx<R>::t *data, int L, int logL, int64_t stride,
                                                   int64_t line_mul, int64_t line_div, int64_t line_mul2,
                                                   const typename Cx<R>::t *tw, int sign) {
  using C2 = typename Cx<R>::t;
  extern __shared__ __align__(16) unsigned char fft_sh[];
  C2 *a = reinterpret_cast<C2 *>(fft_sh), *b = a + L;
  // line index -> base offset: q = hi * line_div + lo  ->  base = hi*line_mul2 + lo*line_mul
  const int64_t q = blockIdx.x;
  const int64_t base = (q / line_div) * line_mul2 + (q % line_div) * line_mul;
  for (int i = threadIdx.x; i < L; i += blockDim.x) a[i] = data[base + (int64_t)i * stride];
  __syncthreads();
  // Stockham autosort: a pass combines sub-transforms of length m = 2^lm
  // into ones of length 2m (radix 2, once when log2 L is odd) or 4m (radix
  // 4): output index (r k) m + j + q m from inputs k m + j + p L / r,
  // twiddled by w_{r m}^{p j} (tw[x] = exp(-2 pi i x / L), conjugated for
  // sign > 0) and combined by the r-point DFT
  int lm = 0;
  if (logL & 1) {
    const int half = L >> 1;
    for (int t = threadIdx.x; t < half; t += blockDim.x) {  // m = 1: no twiddle
      const C2 u = a[t], v = a[t + half];
      b[2 * t] = Cx<R>::mk(u.x + v.x, u.y + v.y);
      b[2 * t + 1] = Cx<R>::mk(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
    C2 *t0 = a;
    a = b;
    b = t0;
    lm = 1;
  }
  const R sg = sign > 0 ? (R)1 : (R)-1;
  for (; lm < logL; lm += 2) {
    const int m = 1 << lm, quarter = L >> 2, tsh = logL - lm - 2;
    for (int t = threadIdx.x; t < quarter; t += blockDim.x) {
      const int j = t & (m - 1), k = t >> lm;
      const C2 a0 = a[t], a1 = a[t + quarter], a2 = a[t + 2 * quarter], a3 = a[t + 3 * quarter];
      C2 w1 = tw[j << tsh], w2 = tw[(2 * j) << tsh], w3 = tw[(3 * j) << tsh];
      if (sign > 0) {
        w1.y = -w1.y;
        w2.y = -w2.y;
        w3.y = -w3.y;
      }
      const C2 c1 = Cx<R>::mk(Cx<R>::fm(a1.x, w1.x, -a1.y * w1.y), Cx<R>::fm(a1.x, w1.y, a1.y * w1.x));
      const C2 c2 = Cx<R>::mk(Cx<R>::fm(a2.x, w2.x, -a2.y * w2.y), Cx<R>::fm(a2.x, w2.y, a2.y * w2.x));
      const C2 c3 = Cx<R>::mk(Cx<R>::fm(a3.x, w3.x, -a3.y * w3.y), Cx<R>::fm(a3.x, w3.y, a3.y * w3.x));
      const C2 t0 = Cx<R>::mk(a0.x + c2.x, a0.y + c2.y), t1 = Cx<R>::mk(a0.x - c2.x, a0.y - c2.y);
      const C2 t2 = Cx<R>::mk(c1.x + c3.x, c1.y + c3.y);
      // (c1 - c3) times w_4 = sign i
      const C2 t3 = Cx<R>::mk(-sg * (c1.y - c3.y), sg * (c1.x - c3.x));
      const int o = (k << (lm + 2)) + j;
      b[o] = Cx<R>::mk(t0.x + t2.x, t0.y + t2.y);
      b[o + m] = Cx<R>::mk(t1.x + t3.x, t1.y + t3.y);
      b[o + 2 * m] = Cx<R>::mk(t0.x - t2.x, t0.y - t2.y);
      b[o + 3 * m] = Cx<R>::mk(t1.x - t3.x, t1.y - t3.y);
    }
    __syncthreads();
    C2 *t0 = a;
    a = b;
    b = t0;
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) data[base + (int64_t)i * stride] = a[i];
}

// tw[k] = exp(-2 pi i k / L), k < L (a radix-4 pass reads up to 3L/4)
__global__ void k_twiddle(double2 *tw, int L) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)L, &s, &c);
  tw[k] = make_double2(c, s);
}

// Embedded kernel c[delta] on the L^d circulant: offsets e in (-s, s) per
// axis, 0 at e = 0 and at the unused index s.
__global__ void k_embed_kernel(double2 *C, int dim, int s, int L, double h, int kind, double w) {
  int64_t tot = 1;
  for (int d = 0; d < dim; d++) tot *= L;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= tot) return;
  int64_t rem = e;
  double r2 = 0.0;
  bool zero = false;
  for (int d = 0; d < dim; d++) {
    int i = (int)(rem % L);
    rem /= L;
    if (i == s) zero = true;
    int off = i < s ? i : i - L;
    r2 += (double)off * off;
  }
  double v = 0.0;
  if (!zero && r2 > 0.0) v = w * kof(kind, r2 * h * h);
  C[e] = make_double2(v, 0.0);
}

// X[grid(i)] = x1[i] + i x2[i] (zero elsewhere); grid(i): linear index of
// point i (caller order) in the s^d grid, embedded in L^d.
template <typename R>
__global__ void k_pack(typename Cx<R>::t *X, const int64_t *gidx, const double *x, int64_t n, int nrhs, int c0,
                       int dim, int s, int L) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t g = gidx[i], pos = 0, mul = 1;
  for (int d = 0; d < dim; d++) {
    pos += (g % s) * mul;
    g /= s;
    mul *= L;
  }
  double re = x[i + (int64_t)c0 * n];
  double im = (c0 + 1 < nrhs) ? x[i + (int64_t)(c0 + 1) * n] : 0.0;
  X[pos] = Cx<R>::mk((R)re, (R)im);
}

template <typename R>
__global__ void k_mul_real(typename Cx<R>::t *X, const typename Cx<R>::t *C, int64_t tot, R scale) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= tot) return;
  const R c = C[e].x * scale;
  X[e] = Cx<R>::mk(X[e].x * c, X[e].y * c);
}

// the FP32 copies of the spectrum and the twiddles, rounded from FP64
__global__ void k_c2_to_f32(float2 *out, const double2 *in, int64_t tot) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= tot) return;
  out[e] = make_float2((float)in[e].x, (float)in[e].y);
}

// y = diag * x + (K x)  for the two packed columns
template <typename R>
__global__ void k_unpack(const typename Cx<R>::t *X, const int64_t *gidx, const double *x, double *y, int64_t n,
                         int nrhs, int c0, int dim, int s, int L, double diag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t g = gidx[i], pos = 0, mul = 1;
  for (int d = 0; d < dim; d++) {
    pos += (g % s) * mul;
    g /= s;
    mul *= L;
  }
  const typename Cx<R>::t v = X[pos];
  y[i + (int64_t)c0 * n] = diag * x[i + (int64_t)c0 * n] + (double)v.x;
  if (c0 + 1 < nrhs) y[i + (int64_t)(c0 + 1) * n] = diag * x[i + (int64_t)(c0 + 1) * n] + (double)v.y;
}

static void fft_nd(double2 *X, int dim, int L, int logL, const double2 *tw, int sign, cudaStream_t st) {
  size_t smem = (size_t)2 * L * sizeof(double2);
  int64_t tot = 1;
  for (int d = 0; d < dim; d++) tot *= L;
  int64_t lines = tot / L;
  for (int ax = 0; ax < dim; ax++) {
    int64_t stride = 1;
    for (int d = 0; d < ax; d++) stride *= L;
    // lines along axis ax: q = hi * stride + lo, lo < stride; base = hi * stride * L + lo
    k_fft_lines<double><<<(unsigned)lines, 256, smem, st>>>(X, L, logL, stride, 1, stride, stride * L, tw, sign); count_launch();
  }
}

// One pass of length-L transforms along axis `ax`, over the lines whose other
// coordinates d lie below lim[d] (lines entirely outside hold zeros, or
// results nobody reads).
template <typename R>
static void fft_pass(typename Cx<R>::t *X, int dim, int L, int logL, const typename Cx<R>::t *tw, int sign, int ax,
                     const int64_t *lim, cudaStream_t st) {
  size_t smem = (size_t)2 * L * sizeof(typename Cx<R>::t);
  int64_t stride[4] = {1, 1, 1, 1};
  for (int d = 0; d < dim; d++) stride[d + 1] = stride[d] * L;
  int o[2] = {-1, -1}, no = 0;
  for (int d = 0; d < dim; d++)
    if (d != ax) o[no++] = d;
  const int64_t lo_lim = no > 0 ? lim[o[0]] : 1, hi_lim = no > 1 ? lim[o[1]] : 1;
  const int64_t mul = no > 0 ? stride[o[0]] : 0, mul2 = no > 1 ? stride[o[1]] : 0;
  const int64_t lines = lo_lim * hi_lim;
  if (lines == 0) return;
  k_fft_lines<R><<<(unsigned)lines, 256, smem, st>>>(X, L, logL, stride[ax], mul, lo_lim, mul2, tw, sign); count_launch();
}

void grid_op_setup(GridOp &G, cudaStream_t st) {
  int64_t tot = 1;
  for (int d = 0; d < G.dim; d++) tot *= G.L;
  cudaFuncSetAttribute(k_fft_lines<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * G.L * (int)sizeof(double2));
  cudaFuncSetAttribute(k_fft_lines<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * G.L * (int)sizeof(float2));
  k_twiddle<<<(G.L + 255) / 256, 256, 0, st>>>(G.tw, G.L); count_launch();
  k_embed_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(G.C, G.dim, G.s, G.L, G.h, G.kind, G.w); count_launch();
  fft_nd(G.C, G.dim, G.L, G.logL, G.tw, -1, st);
}

void grid_op_setup_f32(GridOp &G, cudaStream_t st) {
  int64_t tot = 1;
  for (int d = 0; d < G.dim; d++) tot *= G.L;
  k_c2_to_f32<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(G.Cf, G.C, tot); count_launch();
  k_c2_to_f32<<<(unsigned)((G.L + 255) / 256), 256, 0, st>>>(G.twf, G.tw, G.L); count_launch();
}

template <typename R>
static void grid_op_apply_t(const GridOp &G, typename Cx<R>::t *X, const typename Cx<R>::t *C,
                            const typename Cx<R>::t *tw, const double *x, double *y, int nrhs, cudaStream_t st) {
  int64_t tot = 1;
  for (int d = 0; d < G.dim; d++) tot *= G.L;
  for (int c0 = 0; c0 < nrhs; c0 += 2) {
    cudaMemsetAsync(X, 0, sizeof(typename Cx<R>::t) * tot, st);
    k_pack<R><<<(unsigned)((G.n + 255) / 256), 256, 0, st>>>(X, G.gidx, x, G.n, nrhs, c0, G.dim, G.s, G.L); count_launch();
    // forward: the data sit in [0, s)^d, so an axis not yet transformed
    // limits the lines to its first s coordinates
    int64_t lim[3] = {G.s, G.s, G.s};
    for (int ax = 0; ax < G.dim; ax++) {
      fft_pass<R>(X, G.dim, G.L, G.logL, tw, -1, ax, lim, st);
      lim[ax] = G.L;
    }
    k_mul_real<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, C, tot, (R)(1.0 / (double)tot)); count_launch();
    // inverse, last axis first: only [0, s)^d is read, so an axis already
    // transformed back limits the lines to its first s coordinates
    for (int ax = G.dim - 1; ax >= 0; ax--) {
      for (int d = 0; d < G.dim; d++) lim[d] = d > ax ? G.s : G.L;
      fft_pass<R>(X, G.dim, G.L, G.logL, tw, +1, ax, lim, st);
    }
    k_unpack<R><<<(unsigned)((G.n + 255) / 256), 256, 0, st>>>(X, G.gidx, x, y, G.n, nrhs, c0, G.dim, G.s, G.L,
                                                                G.diag); count_launch();
  }
}

void grid_op_apply(const GridOp &G, const double *x, double *y, int nrhs, cudaStream_t st, bool f32) {
  if (f32)
    grid_op_apply_t<float>(G, G.Xf, G.Cf, G.twf, x, y, nrhs, st);
  else
    grid_op_apply_t<double>(G, G.X, G.C, G.tw, x, y, nrhs, st);
}

// ---------------------------------------------------------------------------
// FP64 vector kernels for the Krylov loop (column-major n x nrhs blocks).
// Reductions are two-pass and deterministic.
// ---------------------------------------------------------------------------

constexpr int RB = 256;      // threads per reduction block
constexpr int RBLK = 240;    // blocks per column in the first pass

// part[(c * nv + i) * RBLK + blk] = partial sum of V_i[:,c] . w[:,c]
__global__ void __launch_bounds__(RB) k_multidot_part(const double *V, int64_t vstride, int nv, const double *w,
                                                      int64_t n, int nrhs, double *part) {
  __shared__ double red[RB / 32];
  const int c = blockIdx.y, i = blockIdx.z, blk = blockIdx.x;
  const double *vi = V + (int64_t)i * vstride + (int64_t)c * n;
  const double *wc = w + (int64_t)c * n;
  double s = 0.0;
  for (int64_t e = blk * (int64_t)RB + threadIdx.x; e < n; e += (int64_t)RB * RBLK) s += vi[e] * wc[e];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < RB / 32 ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) part[((int64_t)c * nv + i) * RBLK + blk] = s;
  }
}

__global__ void k_multidot_final(const double *part, int cnt, double *out) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt) return;
  double s = 0.0;
  for (int b = 0; b < RBLK; b++) s += part[(int64_t)q * RBLK + b];
  out[q] = s;
}

// out[c * nv + i] = V_i[:,c] . w[:,c]
void multidot(const double *V, int64_t vstride, int nv, const double *w, int64_t n, int nrhs, double *part,
              double *out, cudaStream_t st) {
  dim3 g(RBLK, nrhs, nv);
  k_multidot_part<<<g, RB, 0, st>>>(V, vstride, nv, w, n, nrhs, part); count_launch();
  int cnt = nrhs * nv;
  k_multidot_final<<<(cnt + 127) / 128, 128, 0, st>>>(part, cnt, out); count_launch();
}

// y[:,c] = alpha * y[:,c] + sum_i coef[c * nv + i] * V_i[:,c]
__global__ void k_combine(double *y, double alpha, const double *V, int64_t vstride, int nv, const double *coef,
                          int64_t n, int nrhs) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  int c = (int)(e / n);
  double s = alpha * y[e];
  for (int i = 0; i < nv; i++) s += coef[c * nv + i] * V[(int64_t)i * vstride + e];
  y[e] = s;
}

void combine(double *y, double alpha, const double *V, int64_t vstride, int nv, const double *coef, int64_t n,
             int nrhs, cudaStream_t st) {
  int64_t tot = n * nrhs;
  if (tot == 0) return;
  k_combine<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(y, alpha, V, vstride, nv, coef, n, nrhs); count_launch();
}

}  // namespace rss
