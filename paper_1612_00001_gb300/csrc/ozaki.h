// FP64-accurate grouped GEMM on the BF16 tensor cores by exact digit
// splitting (see ozaki.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mbinv {
namespace oz {

constexpr int kDigits = 8;           // balanced base-128 digits of a 56-bit fixed-point entry
constexpr int kMaxKBlocks = 8;       // K blocks of 64 one exact FP32 accumulation may take (K <= 512)
constexpr int kNonFinite = 1 << 30;  // row exponent marking a row that holds Inf or NaN

// Source of one packed operand slab: the rows x cols row-major FP64 matrix
// at src (leading dimension ld), or its transpose (slab row r = column r).
struct PackDesc {
  const double* src;
  int64_t ld;
  int rows, cols;
  int transpose;
  int slab;
};

// One product of a grouped launch:
//     out = beta * Cin + alpha * A_slab * B_slab^T     (FP64, row-major, m x n)
// with alpha = +-1 and beta = 0 or 1 (the Schur products and updates need no
// other; the epilogue then spends one FP64 instruction per entry).
// over the K blocks [kb0, kb0 + nkb) of the slabs.  Cin may be null; it may
// also be out itself (each element is read once, then written).  Rows in
// [nocin_r0, nocin_r1) take no Cin; columns in [skip_c0, skip_c1) are not
// written (the trailing update of a blocked Gauss-Jordan step).
struct Problem {
  int a_slab, b_slab;
  const double* cin;
  int64_t ldcin;
  double* out;
  int64_t ldo;
  int m, n;
  int nocin_r0, nocin_r1;
  int skip_c0, skip_c1;
};

struct Params {
  int kpad;        // padded inner length of the slabs (multiple of tile_k())
  int kb0, nkb;    // K blocks of this launch, nkb <= kMaxKBlocks
  int tiles_m, tiles_n;  // tiles of the largest problem
  double alpha, beta;
  const int* ea;   // row exponents of the A slabs: ea[slab * ea_rows + r]
  const int* eb;   // row exponents of the B slabs: eb[slab * eb_rows + r]
  int ea_rows, eb_rows;
  int* err;        // raised when a bounded wait ran out
  // CTA c takes tiles c, c + grid, ... (CTAs side by side share operand
  // tiles in L2).  1: the grid size is made coprime with tiles_n, so that
  // dead tiles recurring with the column period (skipped columns) fall on
  // every CTA alike instead of on the CTAs whose index shares the period
  int coprime_grid;
  // Test of the timeout path: when nonzero, every CTA first waits this many
  // nanoseconds on a barrier nothing arrives at, raises err and returns
  // before issuing any copy or product (nothing is left in flight).
  unsigned long long stall_ns;
};

// Sets the stall of every later launch_gemm (0 = none); a test hook.
void set_debug_stall(unsigned long long ns);

int tile_m();  // 128 output rows per CTA
int tile_n();  // 64 output columns per CTA
int tile_k();  // 64: inner-dimension tile and padding unit
int pack_rows();  // 32: slab rows are packed in units of this
size_t smem_bytes();

// Packs count slabs: digits dst[((slab * kDigits + p) * rows_pad + r) * kpad + k]
// (p = 0 most significant) and row exponents exps[slab * rows_pad + r].
// Rows and columns beyond the source are written as zeros.
cudaError_t launch_pack(const PackDesc* d_descs, int count, int rows_pad, int kpad, __nv_bfloat16* dst, int* exps,
                        cudaStream_t s);

// One set of slabs to pack (the arguments of launch_pack).
struct PackSet {
  const PackDesc* descs;
  int count;
  int rows_pad;
  __nv_bfloat16* dst;
  int* exps;
};
// Two sets of the same inner length kpad (the two operands of one product)
// in one launch; a set with count 0 is skipped.
cudaError_t launch_pack2(const PackSet& a, const PackSet& b, int kpad, cudaStream_t s);
// a_rows_pad is a multiple of tile_m(), b_rows_pad of tile_n().
cudaError_t launch_gemm(const __nv_bfloat16* apk, int a_slabs, int a_rows_pad, const __nv_bfloat16* bpk, int b_slabs,
                        int b_rows_pad, const Params& P, const Problem* d_probs, int count, cudaStream_t s);

}  // namespace oz
}  // namespace mbinv
