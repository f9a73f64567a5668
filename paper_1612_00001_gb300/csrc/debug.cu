// Test hook of the tensor-core product (not part of the public header): runs
// the grouped tcgen05 GEMM on plain row-major FP32 inputs so that the tests
// can check it against a plain product without going through the recursion.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "tc_gemm.h"

using namespace mbinv;

namespace {

// C[g][r][c] = sum over slices q of slab[g][q][c][r]   (undoes mode 1)
__global__ void unpack_t_kernel(const __nv_bfloat16* pk, int S, int orows, int okpad, float* C, int m, int n) {
  const int g = blockIdx.z, r = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    float x = 0.f;
    for (int q = S - 1; q >= 0; --q) x += __bfloat162float(pk[(((int64_t)g * S + q) * orows + c) * okpad + r]);
    C[((int64_t)g * m + r) * n + c] = x;
  }
}

}  // namespace

extern "C" int mbinv_debug_tc_gemm(const float* A, const float* B, float* C, int m, int n, int k, int S, int count,
                                   int mode, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int T = tc::tile_rows(), KT = tc::tile_k();
  const int mpad = (m + T - 1) / T * T, npad = (n + T - 1) / T * T, kpad = (k + KT - 1) / KT * KT;
  __nv_bfloat16 *apk = nullptr, *bpk = nullptr, *opk = nullptr;
  tc::PackDesc* dd = nullptr;
  tc::TcProblem* dp = nullptr;
  int* derr = nullptr;
  int rc = 0;
  const int okpad = (m + KT - 1) / KT * KT;
  if (cudaMalloc(&apk, (size_t)count * S * mpad * kpad * 2) || cudaMalloc(&bpk, (size_t)count * S * npad * kpad * 2) ||
      cudaMalloc(&opk, (size_t)count * S * npad * (okpad > mpad ? okpad : mpad) * 2) ||
      cudaMalloc(&dd, sizeof(tc::PackDesc) * 2 * count) || cudaMalloc(&dp, sizeof(tc::TcProblem) * count) ||
      cudaMalloc(&derr, sizeof(int)))
    rc = 1;
  if (!rc) {
    std::vector<tc::PackDesc> pd(2 * count);
    std::vector<tc::TcProblem> pr(count);
    for (int g = 0; g < count; ++g) {
      pd[g] = tc::PackDesc{A + (size_t)g * m * k, k, m, k, 0, 0, g};
      pd[count + g] = tc::PackDesc{B + (size_t)g * k * n, n, k, n, 0, 1, g};  // slab row = column of B
      pr[g] = tc::TcProblem{g, g, nullptr, 0, 0, C + (size_t)g * m * n, n, g};
    }
    cudaMemcpyAsync(dd, pd.data(), sizeof(tc::PackDesc) * 2 * count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dp, pr.data(), sizeof(tc::TcProblem) * count, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(derr, 0, sizeof(int), s);
    cudaMemsetAsync(opk, 0, (size_t)count * S * npad * (okpad > mpad ? okpad : mpad) * 2, s);
    if (tc::launch_pack(dd, count, S, mpad, kpad, apk, s) != cudaSuccess) rc = 2;
    if (!rc && tc::launch_pack(dd + count, count, S, npad, kpad, bpk, s) != cudaSuccess) rc = 3;
    tc::TcParams P{};
    P.m = m;
    P.n = n;
    P.kpad = kpad;
    P.tiles_m = mpad / T;
    P.tiles_n = npad / T;
    P.S = S;
    tc::pair_table(S, &P.npairs, P.pa, P.pb);
    P.alpha = 1.f;
    P.beta = 0.f;
    P.mode = mode;
    P.opk = opk;
    P.orows = npad;
    P.okpad = okpad;
    P.err = derr;
    if (!rc && tc::launch_gemm(apk, count, mpad, bpk, count, npad, P, dp, count, s) != cudaSuccess) rc = 4;
    if (!rc && mode == 1) {
      dim3 g((n + 255) / 256, m, count);
      unpack_t_kernel<<<g, 256, 0, s>>>(opk, S, npad, okpad, C, m, n);
    }
    int herr = 0;
    if (!rc && cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = 5;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = 6;
    if (!rc && herr) rc = 7;
  }
  cudaFree(apk);
  cudaFree(bpk);
  cudaFree(opk);
  cudaFree(dd);
  cudaFree(dp);
  cudaFree(derr);
  return rc;
}
