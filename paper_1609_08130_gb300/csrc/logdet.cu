// logdet.cu -- log |det F| of a stored factorization, one value per problem
// (the determinant by-product of Sec. 3.3).
#include <cuda_runtime.h>

#include "internal.h"

namespace rss {

// log|det F| (Sec. 3.3: the triangular factors have unit determinant, so
// det F is the product of the determinants of the boxes' X_RR and of the
// top block): per box, one warp sums log|U_jj| over the diagonal of the LU
// of P X_RR (fixed order); `first` records a DOF id of the box so the host
// can assign it to its problem.  Per problem, one warp sums over the
// diagonal of its top block's LU.
template <typename T>
__global__ void k_logdet_boxes(const FBox<T> *boxes, int nbox, double *part, int64_t *first) {
  const int q = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (q >= nbox) return;
  const FBox<T> &fb = boxes[q];
  const int r = fb.r;
  double s = 0.0;
  for (int j = lane; j < r; j += 32) s += log(fabs((double)fb.LU[(int64_t)j * r + j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    part[q] = s;
    first[q] = fb.b > 0 ? fb.ids[0] : -1;
  }
}

template <typename T> __global__ void k_logdet_top(const T *LU, const int64_t *loff, const int *tn, double *part) {
  const int p = blockIdx.x, lane = threadIdx.x, n = tn[p];
  const T *A = LU + loff[p];
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += log(fabs((double)A[(int64_t)j * n + j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) part[p] = s;
}

template <typename T>
void launch_logdet(const FBox<T> *boxes, int nbox, const T *topLU, const int64_t *loff, const int *tn, int nprob,
                   double *part, int64_t *first, cudaStream_t st) {
  if (nbox > 0) {
    k_logdet_boxes<T><<<(nbox + 7) / 8, 256, 0, st>>>(boxes, nbox, part, first);
    count_launch();
  }
  if (nprob > 0 && topLU) {
    k_logdet_top<T><<<nprob, 32, 0, st>>>(topLU, loff, tn, part + nbox);
    count_launch();
  }
}

template void launch_logdet<float>(const FBox<float> *, int, const float *, const int64_t *, const int *, int,
                                   double *, int64_t *, cudaStream_t);
template void launch_logdet<double>(const FBox<double> *, int, const double *, const int64_t *, const int *, int,
                                    double *, int64_t *, cudaStream_t);

}  // namespace rss
