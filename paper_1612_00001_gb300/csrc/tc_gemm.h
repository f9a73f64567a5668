// Grouped BF16-slice GEMM on tcgen05 tensor cores (see tc_gemm.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mbinv {
namespace tc {

// One problem of a grouped launch.
struct TcProblem {
  int a_slab, b_slab;  // slab indices of its operands in the packed A / B buffers
  const void* cin;     // mode 0: addend (may be null), row-major, FP32 or FP64
  int64_t ldcin;
  int cin_f64;
  void* out;           // mode 0: FP32 output, row-major
  int64_t ldo;
  int out_slab;        // mode 1: slab of the packed output buffer
};

struct TcParams {
  int m, n, kpad;      // output m x n; inner dimension padded to a multiple of 64
  int tiles_m, tiles_n;
  int S;               // slices per operand
  int npairs;          // slice products
  int pa[6], pb[6];    // slice of A / of B of each product
  float alpha, beta;
  int mode;            // 0: out = beta * Cin + alpha * D; 1: slices of alpha * D^T into opk
  __nv_bfloat16* opk;  // mode 1 output buffer [slab][S][orows][okpad]
  int orows, okpad;
  int* err;            // raised when a bounded wait ran out
};

// Source of one packed slab: rows x cols of a row-major FP32/FP64 matrix.
struct PackDesc {
  const void* src;
  int64_t ld;
  int rows, cols;
  int f64;
  int transpose;  // slab row r holds source column r
  int slab;
};

int tile_rows();  // 128: the M and N tile
int tile_k();     // 64: inner-dimension tile and padding unit
size_t smem_bytes();
void pair_table(int S, int* npairs, int* pa, int* pb);

cudaError_t launch_pack(const PackDesc* d_descs, int count, int S, int rows_pad, int kpad, __nv_bfloat16* dst,
                        cudaStream_t s);
cudaError_t launch_gemm(const __nv_bfloat16* apk, int a_slabs, int a_rows_pad, const __nv_bfloat16* bpk, int b_slabs,
                        int b_rows_pad, const TcParams& P, const TcProblem* d_probs, int count, cudaStream_t s);

}  // namespace tc
}  // namespace mbinv
