// common.cuh -- device-side helpers shared by the RS-S kernels.
//
// Scalar type T is double (the plain FP64 form) or float (the mixed form:
// FP32 factor, FP64 residual).  Kernel entries follow the second-kind
// discretisation A = diag*I + w*K (Sec. 1, Eq. 1.3) with the 2D or 3D
// Laplace kernel (Sec. 3.2; Sec. 4, Examples 1 and 2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rss {

constexpr double kPi = 3.14159265358979323846;

// Device error word: the first failing kernel records its code here.
enum DevErr { DERR_NONE = 0, DERR_NUMERIC = 4, DERR_INTERNAL = 7, DERR_CAPACITY = 8 };

__device__ __forceinline__ void set_err(int *err, int code) { atomicCAS(err, 0, code); }

// Division by a loop-invariant divisor 1 <= d < 2^31 with a multiply-high,
// an add and a shift (Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994, Fig. 4.1): with l = ceil(log2 d)
// and m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(m, n) + n) >> l
// for 0 <= n < 2^31.  The index loops that walk a matrix element by
// element use it instead of the hardware-less integer division.
struct FastDiv {
  uint32_t d, m, l;
  __device__ __forceinline__ explicit FastDiv(int dd) : d((uint32_t)dd), l(0) {
    while (l < 31 && (1u << l) < d) l++;
    m = (uint32_t)((((uint64_t)((1ull << l) - d)) << 32) / d) + 1u;
  }
  __device__ __forceinline__ int div(int n) const {
    return (int)((__umulhi(m, (uint32_t)n) + (uint32_t)n) >> l);
  }
  // n = q d + r, 0 <= r < d
  __device__ __forceinline__ void divmod(int n, int &q, int &r) const {
    q = div(n);
    r = n - q * (int)d;
  }
};

// Offsets of the 5^d block around a cell: code = sum_d (delta_d + 2) 5^d.
__host__ __device__ __forceinline__ int code5(int dx, int dy, int dz, int dim) {
  return (dx + 2) + 5 * (dy + 2) + (dim == 3 ? 25 * (dz + 2) : 0);
}
// Offsets of the 3^d block: code = sum_d (delta_d + 1) 3^d.
__host__ __device__ __forceinline__ int code3(int dx, int dy, int dz, int dim) {
  return (dx + 1) + 3 * (dy + 1) + (dim == 3 ? 9 * (dz + 1) : 0);
}
__host__ __device__ __forceinline__ void decode3(int c, int dim, int &dx, int &dy, int &dz) {
  dx = c % 3 - 1;
  dy = (c / 3) % 3 - 1;
  dz = dim == 3 ? c / 9 - 1 : 0;
}

// Points as the kernels see them.  FP64 form: tree-ordered coordinates.
// FP32 form: integer cell index at the finest depth plus an FP32 offset in
// that cell, so differences of nearby points keep full FP32 relative
// accuracy without FP64 arithmetic: x_i - x_j = (c_i - c_j) D + (d_i - d_j).
struct Points {
  const double *x;     // n*dim, tree order
  const int *cell;     // n*3 integer cells at depth 20
  const float *off;    // n*3 offsets in the cell
  float D;             // side of a depth-20 cell
  int dim;
  const double *wdof;  // per-DOF weight w (several problems), or NULL: KernelParams::w
};

template <typename T> struct Dist2;
template <> struct Dist2<double> {
  static __device__ __forceinline__ double eval(const Points &P, int64_t i, int64_t j) {
    const double *a = P.x + i * P.dim, *b = P.x + j * P.dim;
    double dx = a[0] - b[0], dy = a[1] - b[1];
    double r2 = dx * dx + dy * dy;
    if (P.dim == 3) {
      double dz = a[2] - b[2];
      r2 += dz * dz;
    }
    return r2;
  }
};
template <> struct Dist2<float> {
  static __device__ __forceinline__ float eval(const Points &P, int64_t i, int64_t j) {
    const int *ca = P.cell + 3 * i, *cb = P.cell + 3 * j;
    const float *oa = P.off + 3 * i, *ob = P.off + 3 * j;
    float dx = fmaf((float)(ca[0] - cb[0]), P.D, oa[0] - ob[0]);
    float dy = fmaf((float)(ca[1] - cb[1]), P.D, oa[1] - ob[1]);
    float r2 = dx * dx + dy * dy;
    if (P.dim == 3) {
      float dz = fmaf((float)(ca[2] - cb[2]), P.D, oa[2] - ob[2]);
      r2 = fmaf(dz, dz, r2);
    }
    return r2;
  }
};

// K as a function of r^2: kind 0: -log(r)/(2 pi) = -log(r^2)/(4 pi);
// kind 1: 1/(4 pi r).
__device__ __forceinline__ double kof(int kind, double r2) {
  return kind == 0 ? -log(r2) * (1.0 / (4.0 * kPi)) : (1.0 / (4.0 * kPi)) / sqrt(r2);
}
__device__ __forceinline__ float kof(int kind, float r2) {
  return kind == 0 ? -logf(r2) * (float)(1.0 / (4.0 * kPi)) : (float)(1.0 / (4.0 * kPi)) * rsqrtf(r2);
}

struct KernelParams {
  int kind;
  double diag, w;
};

// Matrix entry A_ij = diag (i == j) or w K(x_i - x_j).
template <typename T>
__device__ __forceinline__ T entry(const Points &P, const KernelParams &K, int64_t i, int64_t j) {
  if (i == j) return (T)K.diag;
  const double w = P.wdof ? P.wdof[i] : K.w;
  return (T)w * kof(K.kind, Dist2<T>::eval(P, i, j));
}
// The same with the weight and the diagonal already in T (one problem, no
// per-DOF weights): no FP64 conversion per entry.
template <typename T>
__device__ __forceinline__ T entry_t(const Points &P, int kind, T w, T diag, int64_t i, int64_t j) {
  if (i == j) return diag;
  return w * kof(kind, Dist2<T>::eval(P, i, j));
}

// Weight of the problem a DOF belongs to.
__device__ __forceinline__ double weight_of(const Points &P, const KernelParams &K, int64_t i) {
  return P.wdof ? P.wdof[i] : K.w;
}

// Warp reductions.
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace rss
