// Register-tiled CUDA-core GEMM tile (FP64 DFMA / FP32 FFMA), shared by the
// grouped Schur-product launch and the Gauss-Jordan trailing update.
//
// One CTA of NT = (BM/TM)*(BN/TN) threads computes a BM x BN tile of
// op(A) * op(B) over the K range, staging BK-deep slices of both operands in
// shared memory (double buffered, the next slice is fetched into registers
// while the current one is multiplied).  Each thread owns a TM x TN patch
// held in registers.  Out-of-range elements read as zero, so any m, n, k is
// handled.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mbinv {

template <typename TA, typename TB, typename Acc, int BM, int BN, int BK, int TM, int TN>
struct TileGemm {
  static constexpr int NT = (BM / TM) * (BN / TN);
  static constexpr int TX = BN / TN;  // threads along n
  static constexpr int A_PER = (BM * BK) / NT;
  static constexpr int B_PER = (BK * BN) / NT;
  static_assert((BM * BK) % NT == 0 && (BK * BN) % NT == 0, "tile/thread mismatch");

  // A is stored k-major (a[k][m]); its rows are padded by 16 bytes so that
  // the transposing stores of a row-major A do not all hit one bank.
  static constexpr int PADA = 16 / (int)sizeof(Acc);
  struct Smem {
    Acc a[2][BK][BM + PADA];
    Acc b[2][BK][BN];
  };

  // Loads element e of this thread's share of the A slice starting at k0.
  __device__ __forceinline__ static void load_a(Acc (&ra)[A_PER], const TA* A, int64_t lda, int ta, int m0, int k0,
                                                int M, int K, int tid) {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      const int l = tid + e * NT;
      int r, c;
      if (!ta) { r = l / BK; c = l % BK; } else { c = l / BM; r = l % BM; }
      const int gr = m0 + r, gc = k0 + c;
      Acc v = Acc(0);
      if (gr < M && gc < K) v = (Acc)(ta ? A[(int64_t)gc * lda + gr] : A[(int64_t)gr * lda + gc]);
      ra[e] = v;
    }
  }
  __device__ __forceinline__ static void store_a(Smem& s, int buf, const Acc (&ra)[A_PER], int ta, int tid) {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      const int l = tid + e * NT;
      int r, c;
      if (!ta) { r = l / BK; c = l % BK; } else { c = l / BM; r = l % BM; }
      s.a[buf][c][r] = ra[e];
    }
  }
  __device__ __forceinline__ static void load_b(Acc (&rb)[B_PER], const TB* B, int64_t ldb, int tb, int n0, int k0,
                                                int N, int K, int tid) {
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      const int l = tid + e * NT;
      int r, c;  // r along k, c along n
      if (!tb) { r = l / BN; c = l % BN; } else { c = l / BK; r = l % BK; }
      const int gr = k0 + r, gc = n0 + c;
      Acc v = Acc(0);
      if (gr < K && gc < N) v = (Acc)(tb ? B[(int64_t)gc * ldb + gr] : B[(int64_t)gr * ldb + gc]);
      rb[e] = v;
    }
  }
  __device__ __forceinline__ static void store_b(Smem& s, int buf, const Acc (&rb)[B_PER], int tb, int tid) {
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      const int l = tid + e * NT;
      int r, c;
      if (!tb) { r = l / BN; c = l % BN; } else { c = l / BK; r = l % BK; }
      s.b[buf][r][c] = rb[e];
    }
  }

  // acc[i][j] += sum_k op(A)[m0 + ty*TM + i][k] * op(B)[k][n0 + tx*TN + j]
  __device__ __forceinline__ static void run(Smem& s, const TA* A, int64_t lda, int ta, const TB* B, int64_t ldb,
                                             int tb, int m0, int n0, int M, int N, int K, Acc (&acc)[TM][TN]) {
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    Acc ra[A_PER], rb[B_PER];
    const int nk = (K + BK - 1) / BK;
    if (nk == 0) return;
    load_a(ra, A, lda, ta, m0, 0, M, K, tid);
    load_b(rb, B, ldb, tb, n0, 0, N, K, tid);
    store_a(s, 0, ra, ta, tid);
    store_b(s, 0, rb, tb, tid);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
      const int buf = kt & 1;
      const bool more = kt + 1 < nk;
      if (more) {
        load_a(ra, A, lda, ta, m0, (kt + 1) * BK, M, K, tid);
        load_b(rb, B, ldb, tb, n0, (kt + 1) * BK, N, K, tid);
      }
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        Acc fa[TM], fb[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) fa[i] = s.a[buf][kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) fb[j] = s.b[buf][kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(fa[i], fb[j], acc[i][j]);
      }
      if (more) {
        store_a(s, buf ^ 1, ra, ta, tid);
        store_b(s, buf ^ 1, rb, tb, tid);
      }
      __syncthreads();
    }
  }
};

// Tile configurations per accumulator type.
template <typename Acc>
struct TileCfg;
template <>
struct TileCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};
template <>
struct TileCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};

}  // namespace mbinv
