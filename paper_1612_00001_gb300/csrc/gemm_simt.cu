// Grouped CUDA-core GEMM with a fused epilogue: for every problem g of a
// group, C_g = alpha * op(A_g) op(B_g) + beta * Cin_g.  The Schur products of
// one level of the recursion (Z = P^-1 R and X = K - L Z, Sec. 3.2) go out as
// one launch; each CTA finds its problem by binary search over the problems'
// first tile indices.
#include "mbinv_internal.h"
#include "tile_gemm.cuh"

namespace mbinv {

template <typename TA, typename TB, typename TC, typename Acc>
__global__ void __launch_bounds__(256) gemm_grouped_kernel(const GemmDesc* __restrict__ descs, int ndesc) {
  using Cfg = TileCfg<Acc>;
  using TG = TileGemm<TA, TB, Acc, Cfg::BM, Cfg::BN, Cfg::BK, Cfg::TM, Cfg::TN>;
  __shared__ typename TG::Smem smem;
  const int tile = blockIdx.x;
  int lo = 0, hi = ndesc - 1;
  while (lo < hi) {  // last problem whose tile_start <= tile
    const int mid = (lo + hi + 1) >> 1;
    if (descs[mid].tile_start <= tile) lo = mid; else hi = mid - 1;
  }
  const GemmDesc d = descs[lo];
  const int local = tile - d.tile_start;
  const int m0 = (local / d.tiles_n) * Cfg::BM, n0 = (local % d.tiles_n) * Cfg::BN;
  Acc acc[Cfg::TM][Cfg::TN];
#pragma unroll
  for (int i = 0; i < Cfg::TM; ++i)
#pragma unroll
    for (int j = 0; j < Cfg::TN; ++j) acc[i][j] = Acc(0);
  TG::run(smem, (const TA*)d.A, d.lda, d.ta, (const TB*)d.B, d.ldb, d.tb, m0, n0, d.m, d.n, d.k, acc);
  const int tx = threadIdx.x % TG::TX, ty = threadIdx.x / TG::TX;
  const Acc alpha = (Acc)d.alpha, beta = (Acc)d.beta;
  const TC* cin = (const TC*)d.Cin;
  TC* c = (TC*)d.C;
#pragma unroll
  for (int i = 0; i < Cfg::TM; ++i) {
    const int r = m0 + ty * Cfg::TM + i;
    if (r >= d.m) continue;
#pragma unroll
    for (int j = 0; j < Cfg::TN; ++j) {
      const int q = n0 + tx * Cfg::TN + j;
      if (q >= d.n) continue;
      Acc v = alpha * acc[i][j];
      if (cin != nullptr && beta != Acc(0)) v = fma(beta, (Acc)cin[(int64_t)r * d.ldcin + q], v);
      c[(int64_t)r * d.ldc + q] = (TC)v;
    }
  }
}

void gemm_tile_shape(int combo, int* bm, int* bn) {
  if (combo == G_F32) {
    *bm = TileCfg<float>::BM;
    *bn = TileCfg<float>::BN;
  } else {
    *bm = TileCfg<double>::BM;
    *bn = TileCfg<double>::BN;
  }
}

cudaError_t launch_gemm_grouped(int combo, const GemmDesc* d_descs, int ndesc, int total_tiles, cudaStream_t s) {
  if (ndesc <= 0 || total_tiles <= 0) return cudaSuccess;
  switch (combo) {
    case G_F64: gemm_grouped_kernel<double, double, double, double><<<total_tiles, 256, 0, s>>>(d_descs, ndesc); break;
    case G_F32: gemm_grouped_kernel<float, float, float, float><<<total_tiles, 256, 0, s>>>(d_descs, ndesc); break;
    case G_F32IN_F64: gemm_grouped_kernel<float, float, double, double><<<total_tiles, 256, 0, s>>>(d_descs, ndesc); break;
    case G_F64F32_F64: gemm_grouped_kernel<double, float, double, double><<<total_tiles, 256, 0, s>>>(d_descs, ndesc); break;
    case G_F32F64_F64: gemm_grouped_kernel<float, double, double, double><<<total_tiles, 256, 0, s>>>(d_descs, ndesc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mbinv
