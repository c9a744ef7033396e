// mlp.cu -- the rank-proposal network: a 16-64-64-64-1 tanh perceptron that
// predicts each box's skeleton fraction k / b from the box's size and
// geometry before its ID runs.  The factorization uses the prediction only to
// presize the box's factor storage; the column-pivoted QR still decides the
// rank (Sec. 2.2, Definition 2.1), so a wrong prediction costs memory or a
// retry, never accuracy.  Not part of the paper.
//
// Parameters: one flat FP32 master vector (W1 row-major [64][16], b1, W2
// [64][64], b2, W3 [64][64], b3, w4 [64], b4), and its bfloat16 copy that the
// forward and backward passes read (FP32 arithmetic on the bfloat16 values).
// Training is full-batch Adam: per iteration one fused forward/backward
// launch writing per-CTA gradient partials, a fixed-order reduction, and a
// single-CTA Adam update; the three launches are captured once in a CUDA
// graph and replayed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace rss {

namespace mlpk {

constexpr int NF = MLP_NFEAT, H = MLP_HIDDEN, NP = MLP_NPARAM;
constexpr int OW1 = 0, OB1 = OW1 + H * NF, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H * H,
              OW4 = OB3 + H, OB4 = OW4 + H;
static_assert(OB4 + 1 == NP, "parameter layout");
constexpr int TS = 32;     // samples per tile
constexpr int NTH = 256;   // threads per CTA
constexpr int LDW = H + 1; // padded row of the transposed 64 x 64 weights

// Shared-memory image of the weights, FP32, transposed so that a warp reading
// one input's weights to its 32 consecutive output units is conflict-free,
// and padded so that the backward pass's reads along the other index are too.
struct SW {
  float W1T[NF * H];   // W1T[i*H + j] = W1[j][i]
  float b1[H];
  float W2T[H * LDW];  // W2T[i*LDW + j] = W2[j][i]
  float b2[H];
  float W3T[H * LDW];
  float b3[H];
  float w4[H];
  float b4;
};

struct STile {
  float x[TS * NF];
  float h1[TS * H], h2[TS * H], h3[TS * H];
  float dz[TS * H], dz2[TS * H];
  float o[TS], dout[TS];
};

__device__ void load_weights(SW &s, const __nv_bfloat16 *w) {
  for (int e = threadIdx.x; e < H * NF; e += NTH) {
    int j = e / NF, i = e % NF;
    s.W1T[i * H + j] = __bfloat162float(w[OW1 + e]);
  }
  for (int e = threadIdx.x; e < H * H; e += NTH) {
    int j = e / H, i = e % H;
    s.W2T[i * LDW + j] = __bfloat162float(w[OW2 + e]);
    s.W3T[i * LDW + j] = __bfloat162float(w[OW3 + e]);
  }
  for (int j = threadIdx.x; j < H; j += NTH) {
    s.b1[j] = __bfloat162float(w[OB1 + j]);
    s.b2[j] = __bfloat162float(w[OB2 + j]);
    s.b3[j] = __bfloat162float(w[OB3 + j]);
    s.w4[j] = __bfloat162float(w[OW4 + j]);
  }
  if (threadIdx.x == 0) s.b4 = __bfloat162float(w[OB4]);
}

// out[s][j] = tanh(bias[j] + sum_i WT[i*ld + j] in[s][i]) for the tile's 32
// samples; thread t owns unit j = t % 64 of samples t / 64 + 4 q.
template <int NIN>
__device__ void dense_tanh(const float *WT, int ld, const float *bias, const float *in, float *out) {
  const int j = threadIdx.x & (H - 1), s0 = threadIdx.x >> 6;
  float acc[TS / 4];
#pragma unroll
  for (int q = 0; q < TS / 4; q++) acc[q] = bias[j];
#pragma unroll 4
  for (int i = 0; i < NIN; i++) {
    const float wij = WT[i * ld + j];
#pragma unroll
    for (int q = 0; q < TS / 4; q++) acc[q] = fmaf(wij, in[(s0 + 4 * q) * NIN + i], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < TS / 4; q++) out[(s0 + 4 * q) * H + j] = tanhf(acc[q]);
}

// Forward pass of one tile (x already in t.x); o[s] for every tile slot.
__device__ void tile_forward(const SW &w, STile &t) {
  dense_tanh<NF>(w.W1T, H, w.b1, t.x, t.h1);
  __syncthreads();
  dense_tanh<H>(w.W2T, LDW, w.b2, t.h1, t.h2);
  __syncthreads();
  dense_tanh<H>(w.W3T, LDW, w.b3, t.h2, t.h3);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s = warp; s < TS; s += NTH / 32) {
    float v = t.h3[s * H + lane] * w.w4[lane] + t.h3[s * H + lane + 32] * w.w4[lane + 32];
    v = warp_sum(v);
    if (lane == 0) t.o[s] = v + w.b4;
  }
  __syncthreads();
}

__device__ void load_tile(STile &t, const float *X, int64_t s0, int ns) {
  for (int e = threadIdx.x; e < TS * NF; e += NTH) {
    int s = e / NF;
    t.x[e] = s < ns ? X[(s0 + s) * NF + e % NF] : 0.f;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NTH) k_mlp_fwd(const __nv_bfloat16 *w, const float *X, int64_t n, float *out) {
  extern __shared__ __align__(16) unsigned char smem[];
  SW &sw = *reinterpret_cast<SW *>(smem);
  STile &t = *reinterpret_cast<STile *>(smem + ((sizeof(SW) + 15) & ~size_t(15)));
  load_weights(sw, w);
  __syncthreads();
  const int64_t ntile = (n + TS - 1) / TS;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t s0 = tile * TS;
    const int ns = (int)(n - s0 < TS ? n - s0 : TS);
    load_tile(t, X, s0, ns);
    tile_forward(sw, t);
    if (threadIdx.x < ns) out[s0 + threadIdx.x] = t.o[threadIdx.x];
    __syncthreads();
  }
}

// Fused forward + backward of the mean squared loss over this CTA's tiles;
// the CTA's gradient sum goes to part[blockIdx.x * NP ...] and its sum of
// squared residuals to lpart[blockIdx.x].
__global__ void __launch_bounds__(NTH) k_mlp_grad(const __nv_bfloat16 *w, const float *X, const float *y, int64_t n,
                                                  float *part, double *lpart) {
  extern __shared__ __align__(16) unsigned char smem[];
  SW &sw = *reinterpret_cast<SW *>(smem);
  const size_t o1 = (sizeof(SW) + 15) & ~size_t(15);
  STile &t = *reinterpret_cast<STile *>(smem + o1);
  float *g = reinterpret_cast<float *>(smem + o1 + ((sizeof(STile) + 15) & ~size_t(15)));  // [NP]
  __shared__ double s_loss;
  load_weights(sw, w);
  for (int p = threadIdx.x; p < NP; p += NTH) g[p] = 0.f;
  if (threadIdx.x == 0) s_loss = 0.0;
  __syncthreads();
  const float inv_n = 1.f / (float)n;
  const int tid = threadIdx.x, j = tid & (H - 1), s0l = tid >> 6;
  const int64_t ntile = (n + TS - 1) / TS;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t s0 = tile * TS;
    const int ns = (int)(n - s0 < TS ? n - s0 : TS);
    load_tile(t, X, s0, ns);
    tile_forward(sw, t);
    if (tid < TS) {
      float d = 0.f;
      if (tid < ns) {
        d = t.o[tid] - y[s0 + tid];
        atomicAdd(&s_loss, (double)d * (double)d);  // shared-memory sum; order only affects the loss report
      }
      t.dout[tid] = 2.f * d * inv_n;  // dL/do; zero on padding slots
    }
    __syncthreads();
    // output layer: dz3 = dout * w4 * (1 - h3^2); grads of w4, b4
#pragma unroll
    for (int q = 0; q < TS / 4; q++) {
      const int s = s0l + 4 * q;
      const float h = t.h3[s * H + j];
      t.dz[s * H + j] = t.dout[s] * sw.w4[j] * (1.f - h * h);
    }
    if (tid < H) {
      float a = 0.f;
      for (int s = 0; s < TS; s++) a = fmaf(t.dout[s], t.h3[s * H + tid], a);
      g[OW4 + tid] += a;
    }
    if (tid == H) {
      float a = 0.f;
      for (int s = 0; s < TS; s++) a += t.dout[s];
      g[OB4] += a;
    }
    __syncthreads();
    // layer 3 weights from dz3 and h2; dz2 = (W3^T dz3) * (1 - h2^2)
    for (int e = tid; e < H * H; e += NTH) {
      const int jj = e >> 6, ii = e & 63;
      float a = 0.f;
      for (int s = 0; s < TS; s++) a = fmaf(t.dz[s * H + jj], t.h2[s * H + ii], a);
      g[OW3 + e] += a;
    }
    if (tid < H) {
      float a = 0.f;
      for (int s = 0; s < TS; s++) a += t.dz[s * H + tid];
      g[OB3 + tid] += a;
    }
    {
      float acc[TS / 4];
#pragma unroll
      for (int q = 0; q < TS / 4; q++) acc[q] = 0.f;
      for (int jj = 0; jj < H; jj++) {
        const float wv = sw.W3T[j * LDW + jj];  // W3[jj][j]
#pragma unroll
        for (int q = 0; q < TS / 4; q++) acc[q] = fmaf(wv, t.dz[(s0l + 4 * q) * H + jj], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < TS / 4; q++) {
        const int s = s0l + 4 * q;
        const float h = t.h2[s * H + j];
        t.dz2[s * H + j] = acc[q] * (1.f - h * h);
      }
    }
    __syncthreads();
    // layer 2 weights from dz2 and h1; dz1 = (W2^T dz2) * (1 - h1^2) into dz
    for (int e = tid; e < H * H; e += NTH) {
      const int jj = e >> 6, ii = e & 63;
      float a = 0.f;
      for (int s = 0; s < TS; s++) a = fmaf(t.dz2[s * H + jj], t.h1[s * H + ii], a);
      g[OW2 + e] += a;
    }
    if (tid < H) {
      float a = 0.f;
      for (int s = 0; s < TS; s++) a += t.dz2[s * H + tid];
      g[OB2 + tid] += a;
    }
    {
      float acc[TS / 4];
#pragma unroll
      for (int q = 0; q < TS / 4; q++) acc[q] = 0.f;
      for (int jj = 0; jj < H; jj++) {
        const float wv = sw.W2T[j * LDW + jj];  // W2[jj][j]
#pragma unroll
        for (int q = 0; q < TS / 4; q++) acc[q] = fmaf(wv, t.dz2[(s0l + 4 * q) * H + jj], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < TS / 4; q++) {
        const int s = s0l + 4 * q;
        const float h = t.h1[s * H + j];
        t.dz[s * H + j] = acc[q] * (1.f - h * h);
      }
    }
    __syncthreads();
    // layer 1 weights from dz1 and x
    for (int e = tid; e < H * NF; e += NTH) {
      const int jj = e / NF, ii = e % NF;
      float a = 0.f;
      for (int s = 0; s < TS; s++) a = fmaf(t.dz[s * H + jj], t.x[s * NF + ii], a);
      g[OW1 + e] += a;
    }
    if (tid < H) {
      float a = 0.f;
      for (int s = 0; s < TS; s++) a += t.dz[s * H + tid];
      g[OB1 + tid] += a;
    }
    __syncthreads();
  }
  for (int p = tid; p < NP; p += NTH) part[(int64_t)blockIdx.x * NP + p] = g[p];
  if (tid == 0) lpart[blockIdx.x] = s_loss;
}

// grad[p] = sum over CTAs in index order (deterministic); loss = mean squared
// residual.
__global__ void k_mlp_reduce(const float *part, const double *lpart, int nblk, int64_t n, float *grad,
                             double *loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NP) {
    float a = 0.f;
    for (int b = 0; b < nblk; b++) a += part[(int64_t)b * NP + p];
    grad[p] = a;
  }
  if (p == 0) {
    double l = 0.0;
    for (int b = 0; b < nblk; b++) l += lpart[b];
    *loss = l / (double)n;
  }
}

// One Adam step on the FP32 master parameters, then their bfloat16 copy.
// The step counter lives in device memory so a captured graph replays
// unchanged.
__global__ void __launch_bounds__(1024) k_mlp_adam(float *theta, float *m, float *v, const float *grad,
                                                   __nv_bfloat16 *wbf, int *step, float lr, float beta1,
                                                   float beta2, float eps) {
  const int t = *step + 1;
  const float bc1 = 1.f - powf(beta1, (float)t), bc2 = 1.f - powf(beta2, (float)t);
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    const float gp = grad[p];
    const float mp = beta1 * m[p] + (1.f - beta1) * gp;
    const float vp = beta2 * v[p] + (1.f - beta2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float th = theta[p] - lr * (mp / bc1) / (sqrtf(vp / bc2) + eps);
    theta[p] = th;
    wbf[p] = __float2bfloat16_rn(th);
  }
  __syncthreads();
  if (threadIdx.x == 0) *step = t;
}

__global__ void k_mlp_round(const float *theta, __nv_bfloat16 *wbf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NP) wbf[p] = __float2bfloat16_rn(theta[p]);
}

size_t fwd_smem() { return ((sizeof(SW) + 15) & ~size_t(15)) + sizeof(STile); }
size_t grad_smem() {
  return ((sizeof(SW) + 15) & ~size_t(15)) + ((sizeof(STile) + 15) & ~size_t(15)) + sizeof(float) * NP;
}

}  // namespace mlpk

void mlp_round(const float *theta, void *wbf, cudaStream_t st) {
  mlpk::k_mlp_round<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(theta, (__nv_bfloat16 *)wbf);
  count_launch();
}

void mlp_forward(const void *wbf, const float *X, int64_t n, float *out, cudaStream_t st) {
  if (n <= 0) return;
  const size_t sm = mlpk::fwd_smem();
  cudaFuncSetAttribute(mlpk::k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int64_t ntile = (n + mlpk::TS - 1) / mlpk::TS;
  const int grid = (int)std::min<int64_t>(ntile, 2 * 152);
  mlpk::k_mlp_fwd<<<grid, mlpk::NTH, sm, st>>>((const __nv_bfloat16 *)wbf, X, n, out);
  count_launch();
}

int mlp_grad_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + mlpk::TS - 1) / mlpk::TS, 152)); }

void mlp_gradient(const void *wbf, const float *X, const float *y, int64_t n, float *part, double *lpart, float *grad,
                  double *loss, cudaStream_t st) {
  const size_t sm = mlpk::grad_smem();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  if (cap == cudaStreamCaptureStatusNone)  // set once outside the captured training step
    cudaFuncSetAttribute(mlpk::k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int nblk = mlp_grad_blocks(n);
  mlpk::k_mlp_grad<<<nblk, mlpk::NTH, sm, st>>>((const __nv_bfloat16 *)wbf, X, y, n, part, lpart);
  mlpk::k_mlp_reduce<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(part, lpart, nblk, n, grad, loss);
  count_launch(2);
}

void mlp_adam(float *theta, float *m, float *v, const float *grad, void *wbf, int *step, float lr,
              cudaStream_t st) {
  mlpk::k_mlp_adam<<<1, 1024, 0, st>>>(theta, m, v, grad, (__nv_bfloat16 *)wbf, step, lr, 0.9f, 0.999f, 1e-8f);
  count_launch();
}

}  // namespace rss
