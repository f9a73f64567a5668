// Grouped BF16 GEMM on the fifth-generation tensor cores (tcgen05, sm_103a).
//
// For every problem g of a launch
//     D_g = sum over slice pairs (s, t) of A_g^(s) * B_g^(t)^T      (FP32)
// where A^(s) / B^(t) are BF16 slices of FP32 operands (x = s0 + s1 + s2,
// each slice the BF16 rounding of what the previous ones leave), stored
// K-major in packed slabs [slab][slice][rows][kpad].  One CTA computes one
// 128 x 128 output tile:
//   warp 0, one lane:  TMA producer - 3-D tiled bulk copies (128B swizzle) of
//                      the A and B K-slices into a STAGES-deep smem ring;
//   warp 1:            allocates 128 TMEM columns; one lane issues
//                      tcgen05.mma (M=128, N=128, K=16, BF16 in, FP32 acc)
//                      and frees ring slots with tcgen05.commit;
//   warps 0-3:         epilogue - tcgen05.ld of the accumulator (one TMEM
//                      lane per output row) fused with the Schur update:
//                      mode 0:  out = beta * Cin + alpha * D  (FP32, row-major)
//                      mode 1:  the BF16 slices of D^T written straight into
//                               the packed operand slab of the next product.
// Every wait on an mbarrier is bounded (about two seconds of %globaltimer);
// a wait that runs out raises the error word, and the CTA drains, frees its
// TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>

#include "mbinv_internal.h"
#include "tc_gemm.h"
#include "tcgen05_ptx.cuh"

namespace mbinv {
namespace tc {

namespace {

using namespace mbinv::ptx;

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int STAGES = 3;  // 97 KB of shared memory: two CTAs per SM overlap epilogue and main loop
constexpr int THREADS = 128;
constexpr uint32_t TILE_A_BYTES = BM * BK * 2;  // 16 KB
constexpr uint32_t TILE_B_BYTES = BN * BK * 2;  // 16 KB
constexpr uint32_t TMEM_COLS = 128;
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(THREADS, 2)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcParams P, const TcProblem* __restrict__ probs) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + STAGES * TILE_A_BYTES;
  uint64_t* full = (uint64_t*)(sB + STAGES * TILE_B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* failed = (int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_per = P.tiles_m * P.tiles_n;
  const int g = blockIdx.x / tiles_per;
  const int rem = blockIdx.x - g * tiles_per;
  const int tm = rem / P.tiles_n, tn = rem - (rem / P.tiles_n) * P.tiles_n;
  const TcProblem pr = probs[g];

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nkb = P.kpad / BK;
  const int nk = P.npairs * nkb;
  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (kt >= STAGES && !mbar_wait(&empty[s], ph ^ 1u)) {
        atomicExch(failed, 1);
        break;
      }
      if (*(volatile int*)failed) break;
      mbar_expect_tx(&full[s], TILE_A_BYTES + TILE_B_BYTES);
      const int pq = kt / nkb, kb = kt - pq * nkb;
      tma_load_3d(sA + s * TILE_A_BYTES, &tmA, &full[s], kb * BK, tm * BM, pr.a_slab * P.S + P.pa[pq]);
      tma_load_3d(sB + s * TILE_B_BYTES, &tmB, &full[s], kb * BK, tn * BN, pr.b_slab * P.S + P.pb[pq]);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    int issued = 0;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        atomicExch(failed, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA + s * TILE_A_BYTES), b0 = smem_u32(sB + s * TILE_B_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        umma(tmem, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), (kt > 0 || kk > 0) ? 1u : 0u);
      }
      umma_commit(&empty[s]);
      ++issued;
    }
    umma_commit(done);  // arrives when every MMA issued above has completed
    (void)issued;
  }
  __syncwarp();

  // ---------------- epilogue (all four warps; warp w owns TMEM lanes 32w..32w+31)
  bool ok = mbar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok || *(volatile int*)failed) {
    if (lane == 0 && P.err) atomicExch(P.err, 1);
  } else {
    const int row = tm * BM + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(trow + c0, v);
      if (P.mode == 0) {
        // stage the warp's 32 x 16 piece through shared memory (the ring is
        // free once every MMA has completed) so that each row is read and
        // written as one contiguous segment by consecutive lanes
        float* T = (float*)base + warp * (32 * 17);
#pragma unroll
        for (int t = 0; t < 16; ++t) T[lane * 17 + t] = v[t];
        __syncwarp();
        const int rr = lane >> 4, cc = lane & 15;  // two rows of 16 columns per pass
        const int col = tn * BN + c0 + cc;
#pragma unroll 4
        for (int r2 = 0; r2 < 32; r2 += 2) {
          const int lr = r2 + rr;
          const int grow = tm * BM + warp * 32 + lr;
          if (grow < P.m && col < P.n) {
            // FP32 epilogue: the output is FP32, and FP64 arithmetic is scarce here
            float y = P.alpha * T[lr * 17 + cc];
            if (pr.cin) {
              const float ci = pr.cin_f64 ? (float)((const double*)pr.cin)[(int64_t)grow * pr.ldcin + col]
                                          : ((const float*)pr.cin)[(int64_t)grow * pr.ldcin + col];
              y = fmaf(P.beta, ci, y);
            }
            ((float*)pr.out)[(int64_t)grow * pr.ldo + col] = y;
          }
        }
        __syncwarp();
      } else {
        // D^T slices into the packed K-major slab of the next product:
        // element (n, k) of slab [out_slab][q] is D[k][n]
        if (row < P.okpad) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int col = tn * BN + c0 + t;
            if (col < P.orows) {
              __nv_bfloat16 sl[3];
              split_bf16(P.alpha * v[t], P.S, sl);
              for (int q = 0; q < P.S; ++q) {
                const int64_t idx = (((int64_t)pr.out_slab * P.S + q) * P.orows + col) * P.okpad + row;
                P.opk[idx] = sl[q];
              }
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// packed slab [slab][q][rows_pad][kpad] <- slices of src (rows x cols, ld), or
// of its transpose (output row r = source column r).
__global__ void pack_kernel(const PackDesc* __restrict__ descs, int S, int rows_pad, int kpad, __nv_bfloat16* dst) {
  const PackDesc d = descs[blockIdx.z];
  const int r = blockIdx.y;  // output row
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < kpad; c += gridDim.x * blockDim.x) {
    float x = 0.f;
    // output element (r, c): source (r, c) or (c, r)
    const int sr = d.transpose ? c : r, sc = d.transpose ? r : c;
    if (sr < d.rows && sc < d.cols) {
      const int64_t idx = (int64_t)sr * d.ld + sc;
      x = d.f64 ? (float)((const double*)d.src)[idx] : ((const float*)d.src)[idx];
    }
    __nv_bfloat16 sl[3];
    split_bf16(x, S, sl);
    for (int q = 0; q < S; ++q) dst[(((int64_t)d.slab * S + q) * rows_pad + r) * kpad + c] = sl[q];
  }
}

}  // namespace

int tile_rows() { return BM; }
int tile_k() { return BK; }

size_t smem_bytes() { return STAGES * (TILE_A_BYTES + TILE_B_BYTES) + 1024 + 256; }

void pair_table(int S, int* npairs, int* pa, int* pb) {
  // slice pairs (s, t) with s + t < S, smallest products first
  int n = 0;
  for (int sum = S - 1; sum >= 0; --sum)
    for (int s = sum; s >= 0; --s) {
      pa[n] = s;
      pb[n] = sum - s;
      ++n;
    }
  *npairs = n;
}

cudaError_t launch_pack(const PackDesc* d_descs, int count, int S, int rows_pad, int kpad, __nv_bfloat16* dst,
                        cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  dim3 grid((kpad + 255) / 256, rows_pad, count);
  pack_kernel<<<grid, 256, 0, s>>>(d_descs, S, rows_pad, kpad, dst);
  return cudaGetLastError();
}

cudaError_t launch_gemm(const __nv_bfloat16* apk, int a_slabs, int a_rows_pad, const __nv_bfloat16* bpk, int b_slabs,
                        int b_rows_pad, const TcParams& P, const TcProblem* d_probs, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (P.kpad % BK || a_rows_pad % BM || b_rows_pad % BN || P.tiles_m * BM > a_rows_pad ||
      P.tiles_n * BN > b_rows_pad)
    return cudaErrorInvalidValue;
  if (((uintptr_t)apk | (uintptr_t)bpk) & 15) return cudaErrorInvalidValue;
  CUtensorMap ta, tb;
  if (!make_map(&ta, apk, P.kpad, a_rows_pad, a_slabs * P.S, BM)) return cudaErrorInvalidValue;
  if (!make_map(&tb, bpk, P.kpad, b_rows_pad, b_slabs * P.S, BN)) return cudaErrorInvalidValue;
  const size_t sm = smem_bytes();
  {
    cudaError_t e = once_per_device((const void*)tc_gemm_kernel, [sm] {
      return cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    });
    if (e != cudaSuccess) return e;
  }
  const int grid = count * P.tiles_m * P.tiles_n;
  tc_gemm_kernel<<<grid, THREADS, sm, s>>>(ta, tb, P, d_probs);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace mbinv
