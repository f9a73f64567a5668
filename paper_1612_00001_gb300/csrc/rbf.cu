// The LS-SVM matrix of Sec. 7 (Eq. A) as a block producer for contexts that
// do not store M:
//     A_gamma = [[0, 1^T], [1, K + I / gamma]],  K_pq = exp(-|x_p - x_q|^2 / (2 sigma^2)),
// of order n + 1, row and column 0 being the border.  Each entry is computed
// in FP64 from the points, which are the only thing stored.
#include <cuda_runtime.h>

#include "../../include/mbinv.h"
#include "mbinv_internal.h"

namespace mbinv {
namespace {

// One thread per entry of the requested block; the dim coordinates of both
// points are read from L1/L2 (dim is small next to the block).
template <typename T>
__global__ void rbf_block_kernel(const double* __restrict__ x, int64_t npts, int64_t dim, double inv2s2, double ridge,
                                 int64_t r0, int64_t c0, int64_t rows, int64_t cols, T* __restrict__ dst,
                                 int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = r0 + e / cols, c = c0 + e % cols;
  double v;
  if (r == 0 && c == 0) {
    v = 0.0;
  } else if (r == 0 || c == 0) {
    v = 1.0;
  } else {
    const double* xp = x + (r - 1) * dim;
    const double* xq = x + (c - 1) * dim;
    double d2 = 0.0;
    for (int64_t t = 0; t < dim; ++t) {
      const double d = xp[t] - xq[t];
      d2 += d * d;
    }
    v = exp(-d2 * inv2s2) + (r == c ? ridge : 0.0);
  }
  dst[(e / cols) * ldd + e % cols] = (T)v;
}

}  // namespace
}  // namespace mbinv

extern "C" int mbinv_rbf_block(int64_t r0, int64_t c0, int64_t rows, int64_t cols, void* dst, int64_t ldd, int dtype,
                               void* stream, void* user) {
  const mbinv_rbf* p = (const mbinv_rbf*)user;
  if (!p || !p->x || !dst || p->n <= 0 || p->dim <= 0 || !(p->sigma > 0.0) || !(p->gamma > 0.0) || r0 < 0 ||
      c0 < 0 || rows < 0 || cols < 0 || r0 + rows > p->n + 1 || c0 + cols > p->n + 1 || ldd < cols)
    return 1;
  const int64_t nel = rows * cols;
  if (nel == 0) return 0;
  const unsigned blocks = (unsigned)((nel + 255) / 256);
  const double inv2s2 = 1.0 / (2.0 * p->sigma * p->sigma), ridge = 1.0 / p->gamma;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == mbinv::F64)
    mbinv::rbf_block_kernel<double><<<blocks, 256, 0, s>>>(p->x, p->n, p->dim, inv2s2, ridge, r0, c0, rows, cols,
                                                            (double*)dst, ldd);
  else if (dtype == mbinv::F32)
    mbinv::rbf_block_kernel<float><<<blocks, 256, 0, s>>>(p->x, p->n, p->dim, inv2s2, ridge, r0, c0, rows, cols,
                                                           (float*)dst, ldd);
  else
    return 1;
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
