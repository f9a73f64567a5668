// FP64-accurate grouped GEMM on the BF16 tensor cores (tcgen05, sm_103a), by
// exact digit splitting - the error-free splitting idea of Ozaki, Ogita,
// Oishi and Rump, here with integer digits.
//
// Packing.  Every entry x of row r of an operand is written, relative to the
// power of two 2^E_r just above the row's largest magnitude, as a 56-bit
// fixed-point integer and its balanced base-128 digits:
//     X = round(x * 2^(55 - E_r)) = sum_{p=0..7} d_p * 128^(7 - p),  |d_p| <= 64,
// all exact in BF16.  The rounding error is at most 2^(E_r - 56).
//
// Product.  For C = A * B^T (B packed by rows of B^T, i.e. transposed)
//     sum_k X_ik Y_jk = sum_{p,q} 128^(14 - p - q) * G_{p+q},
//     G_g = sum_k sum_{p+q=g} d_p(i,k) e_q(j,k).
// Each digit product is an integer of at most 2^12, so G_g (at most 8 pairs,
// K <= 512 terms) stays within 2^24 and the FP32 accumulators of
// tcgen05.mma hold it exactly.  The 36 pairs with g <= 7 are kept; the
// dropped ones weigh at most 2^-53 K max|a_i.| max|b_j.| - the size of an
// FP64 product's own rounding error.  Then
//     C_ij = 2^(E_i + F_j - 61) * S,  S = sum_{g=0..7} G_g 128^(7 - g),
// where S (below 2^75) is formed in integer arithmetic and rounded once to
// FP64; the Schur update out = beta * Cin + alpha * C takes one more FP64
// rounding.  GB300's FP64 pipe is narrow, so the epilogue does everything but
// that last add with integer instructions.
//
// Kernel.  Persistent: one CTA per SM (the eight 64-column group
// accumulators take all 512 TMEM columns) walks the 128 x 64 output tiles of
// the launch, with three roles:
//   warp 0, one lane:  TMA producer.  Per pass and K block of 64 it loads
//                      the B digits of the pass (0-3 or 0-7, 3-D copies of
//                      four digits, 32 KB each; double buffered) and the A
//                      digits of the pass (0-3 or 0-7, 16 KB each) into a
//                      four-deep ring; it runs ahead into the next tile while
//                      the current one is read out.
//   warp 1, one lane:  MMA issuer, two passes per tile.  Pass 0: the pairs
//                      with p + q <= 3 (groups 0-3, TMEM columns 0-255);
//                      pass 1: the others (groups 4-7, columns 256-511).  One
//                      tcgen05.mma per A digit and pass multiplies it by the
//                      B digits q of that pass stacked along N, writing TMEM
//                      columns 64 (p + q) - so every pair lands in its group
//                      G_{p+q} without any data movement.  A pass starts once
//                      the epilogue has read its half of the previous tile
//                      out, so each half's read-out overlaps the other's MMAs.
//   warps 2-17:        epilogue.  Warp w reads TMEM lanes 32 (w mod 4) ..
//                      (a row per thread) and one quarter of the columns, one
//                      half of the groups after each pass, combines them into
//                      registers, hands each half back to the MMA warp, then
//                      reads Cin and writes beta * Cin + alpha * C (16
//                      contiguous entries per thread) while the next tile's
//                      MMAs run.
// Every mbarrier wait is bounded (about two seconds of %globaltimer); a wait
// that runs out raises the error word and the CTA drains, frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "mbinv_internal.h"
#include "ozaki.h"
#include "tcgen05_ptx.cuh"

namespace mbinv {
namespace oz {

namespace {

using namespace mbinv::ptx;

constexpr int ND = kDigits;
constexpr int BM = 128, BN = 64, BK = 64;
constexpr int ASTAGES = 4;
constexpr int NEPI = 16;                  // epilogue warps: 4 lane quarters x 4 column quarters
constexpr int THREADS = 64 + 32 * NEPI;   // producer warp, MMA warp, epilogue warps
constexpr int PR = 16;                                  // slab rows per pack CTA
constexpr int PKC = 512;                                // K entries a pack CTA stages at a time
constexpr int PMAXR = 64;                               // most slab rows per pack CTA
constexpr int kPackSmemMax = 68 * 1024;                 // bound on rpc * (kc + 1) doubles
constexpr uint32_t A_BYTES = BM * BK * 2;               // one digit of the A tile: 16 KB
constexpr uint32_t BQ_BYTES = BN * BK * 2;              // one digit of the B tile: 8 KB
constexpr uint32_t B_BYTES = ND * BQ_BYTES;             // all digits of the B tile: 64 KB
constexpr uint32_t TMEM_COLS = 512;

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}

// Balanced base-128 digits of round(x * 2^(55 - E)), with 2^E > |x|; zero
// and subnormal x give zero digits.  Integer instructions only.
__device__ __forceinline__ void digits8(double x, int E, int (&d)[ND]) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  int64_t X = 0;
  if (ex != 0 && E < kNonFinite) {
    const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // x = m 2^(ex - 1075)
    const int sh = ex - 1020 - E;                                   // X = m 2^sh, sh <= 2
    uint64_t u = 0;
    if (sh >= 0) {
      u = m << sh;
    } else if (sh >= -54) {
      const int r = -sh;
      u = (m + (1ull << (r - 1))) >> r;  // nearest, ties away from zero
    }
    X = (bits >> 63) ? -(int64_t)u : (int64_t)u;
  }
  // The balanced digits (d_1..d_7 in [-64, 63]) are the base-128 digits of
  // X + B, B = 64 (1 + 128 + ... + 128^7), each less 64: X + B lies in
  // (0, 2^57) for |X| <= 2^55, and every digit comes from its own shift.
  constexpr long long kBias = 64LL * (((1LL << 56) - 1) / 127);
  const uint64_t Y = (uint64_t)(X + kBias);
  d[0] = (int)(Y >> 49) - 64;
#pragma unroll
  for (int p = 1; p < ND; ++p) d[p] = (int)((Y >> (7 * (ND - 1 - p))) & 127u) - 64;
}

// 8-byte asynchronous copy global -> shared; ok = false writes zeros and
// reads nothing.
__device__ __forceinline__ void cp_async8(void* dst, const double* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(ok ? 8 : 0)
               : "memory");
}

// The BF16 pair of two digits (|d| <= 64: exact in BF16): each digit becomes
// an FP32 through the mantissa of 1.5 * 2^23 (integer add, FP32 subtract).
__device__ __forceinline__ __nv_bfloat162 digit_pair(int a, int b) {
  const float fa = __int_as_float(0x4B400000 + a) - 12582912.0f;
  const float fb = __int_as_float(0x4B400000 + b) - 12582912.0f;
  return __floats2bfloat162_rn(fa, fb);
}

// The rare results below the normal range or above it: mant 2^(e2 - 52),
// through the FP64 pipe (kept out of line so that the common path issues no
// FP64 instruction).
__device__ __noinline__ double scale_rare(uint64_t mant, int e2, bool neg) {
  const double v = scalbn((double)mant, e2 - 52);
  return neg ? -v : v;
}

// r += b for 96-bit two's-complement integers held as three 32-bit limbs
// (one carry chain).
__device__ __forceinline__ void add96(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t b0, uint32_t b1,
                                      uint32_t b2) {
  asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
      : "+r"(r0), "+r"(r1), "+r"(r2)
      : "r"(b0), "r"(b1), "r"(b2));
}

// +-2^e * S with S = sum_g a_g 128^(7 - g), rounded once to FP64 (ties to
// even), negated when neg_alpha; 32-bit integer instructions only (carry
// chains in place of 64-bit arithmetic), the exponent field assembled
// directly.  Group g sums g + 1 digit pairs over at most 512 terms, so
// |a_g| <= (g + 1) 2^21 and |S| < 2^75.  With the Horner pairs
// h0 = a_0 128 + a_1, h1, l0, l1 (each below 2^31 in magnitude by that bound)
//     S = h0 2^42 + h1 2^28 + l0 2^14 + l1,
// summed as a 96-bit integer in three 32-bit limbs, then taken to sign and
// magnitude, whose leading 53 bits are rounded with the bits below them.
__device__ __forceinline__ double combine(int h0, int h1, int l0, int l1, int e, bool neg_alpha) {
  uint32_t s0 = (uint32_t)l1, s1 = (uint32_t)(l1 >> 31), s2 = s1;
  add96(s0, s1, s2, (uint32_t)l0 << 14, (uint32_t)(l0 >> 18), (uint32_t)(l0 >> 31));
  add96(s0, s1, s2, (uint32_t)h1 << 28, (uint32_t)(h1 >> 4), (uint32_t)(h1 >> 31));
  add96(s0, s1, s2, 0u, (uint32_t)h0 << 10, (uint32_t)(h0 >> 22));
  const uint32_t sg = (uint32_t)((int)s2 >> 31);  // all ones when S < 0
  uint32_t m0 = s0 ^ sg, m1 = s1 ^ sg, m2 = s2 ^ sg;
  add96(m0, m1, m2, sg & 1u, 0u, 0u);  // |S|
  if ((m0 | m1 | m2) == 0u) return 0.0;
  const int top = m2 ? 95 - __clz((int)m2) : (m1 ? 63 - __clz((int)m1) : 31 - __clz((int)m0));  // <= 74
  uint32_t mh, ml;  // the significand, leading bit at bit 52 of mh:ml (bit 53 after a carry)
  if (top <= 52) {  // exact: shift up
    const int k = 52 - top;
    if (k >= 32) {
      mh = m0 << (k - 32);
      ml = 0u;
    } else {
      mh = __funnelshift_l(m0, m1, k);
      ml = m0 << k;
    }
  } else {  // sh = top - 52 <= 22 bits rounded off
    const int sh = top - 52;
    ml = __funnelshift_r(m0, m1, sh);
    mh = __funnelshift_r(m1, m2, sh);
    const uint32_t rem = m0 & ((1u << sh) - 1u), half = 1u << (sh - 1);
    const uint32_t up = (rem > half || (rem == half && (ml & 1u))) ? 1u : 0u;
    asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+r"(ml), "+r"(mh) : "r"(up));
  }
  const bool neg_out = (sg != 0u) != neg_alpha;
  const int e2 = top + e;  // value = mant 2^(e2 - 52)
  const int e2n = e2 + (int)(mh >> 21);
  if (e2n < -1022 || e2n > 1023) return scale_rare(((uint64_t)mh << 32) | ml, e2, neg_out);
  // a carry out of the rounding leaves 2^53, whose low 52 bits are zero
  const uint32_t hi = ((uint32_t)neg_out << 31) | ((uint32_t)(e2n + 1023) << 20) | (mh & 0xFFFFFu);
  return __hiloint2double((int)hi, (int)ml);
}

// Decodes grid tile t: problem g, row tile tm, column tile tn; false when the
// tile lies past its problem's extent or wholly inside its skipped columns.
__device__ __forceinline__ bool tile_live(const Params& P, const Problem* __restrict__ probs, int t, int* g, int* tm,
                                          int* tn) {
  const int tiles_per = P.tiles_m * P.tiles_n;
  *g = t / tiles_per;
  const int rem = t - *g * tiles_per;
  *tm = rem / P.tiles_n;
  *tn = rem - *tm * P.tiles_n;
  const Problem& pr = probs[*g];
  return !(*tm * BM >= pr.m || *tn * BN >= pr.n || (*tn * BN >= pr.skip_c0 && *tn * BN + BN <= pr.skip_c1));
}

// The first nq (4 or 8) digits of the B tile of one K block into the next of
// two buffers.
__device__ __forceinline__ bool load_b_block(uint8_t* sB, uint64_t* fullB, uint64_t* emptyB, const CUtensorMap* tmB,
                                             int* nbq, int kb, int tn, int bslab, int nq) {
  const int s = *nbq & 1;
  if (*nbq >= 2 && !mbar_wait(&emptyB[s], ((uint32_t)(*nbq >> 1) & 1u) ^ 1u)) return false;
  mbar_expect_tx(&fullB[s], nq * BQ_BYTES);
  for (int h = 0; h < nq; h += 4)  // the map's box holds four digits
    tma_load_3d(sB + s * B_BYTES + h * BQ_BYTES, tmB, &fullB[s], kb * BK, tn * BN, bslab * ND + h);
  ++*nbq;
  return true;
}

__global__ void __launch_bounds__(THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Params P,
                   const Problem* __restrict__ probs, int total_tiles) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sB = base;                          // 2 x 64 KB
  uint8_t* sA = base + 2 * B_BYTES;            // ASTAGES x 16 KB
  uint64_t* fullB = (uint64_t*)(sA + ASTAGES * A_BYTES);
  uint64_t* emptyB = fullB + 2;
  uint64_t* fullA = emptyB + 2;
  uint64_t* emptyA = fullA + ASTAGES;
  // The 36 digit pairs run in two passes per tile: pass 0 the pairs with
  // p + q <= 3 (groups 0-3, TMEM columns 0-255), pass 1 the others (groups
  // 4-7, columns 256-511); each half of TMEM is filled and handed back on its
  // own, so the epilogue reads one half while the MMAs fill the other.
  uint64_t* tfull = emptyA + ASTAGES;   // [2] a half's accumulators complete (MMA -> epilogue)
  uint64_t* tempty = tfull + 2;         // [2] a half read out (epilogue -> MMA)
  uint64_t* stall = tempty + 2;         // test of the timeout path: never arrived at
  uint32_t* tmem_slot = (uint32_t*)(stall + 1);
  int* failed = (int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&fullB[s], 1);
      mbar_init(&emptyB[s], 1);
    }
    for (int s = 0; s < ASTAGES; ++s) {
      mbar_init(&fullA[s], 1);
      mbar_init(&emptyA[s], 1);
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(&tfull[h], 1);
      mbar_init(&tempty[h], NEPI);
    }
    mbar_init(stall, 1);
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
  if (P.stall_ns) {
    // nothing arrives at `stall`: the wait runs out, the CTA raises the
    // error word and every role below finds `failed` set before it issues
    // anything
    if (threadIdx.x == 0 && !mbar_wait_ns(stall, 0, P.stall_ns)) {
      *failed = 1;
      if (P.err) atomicExch(P.err, 1);
    }
    __syncthreads();
  }
  const bool stalled = *(volatile int*)failed != 0;

  if (stalled) {
    // skip every role
  } else if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: runs ahead into the next tile while the
      // epilogue of the current one drains the accumulators.  Per tile and
      // pass the K blocks in order: B digits 0-3 (pass 0) or 0-7 (pass 1),
      // and A digits 0-3 (pass 0) or 0-7 (pass 1).
      int na = 0, nbq = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < total_tiles; t += gridDim.x) {
        int g, tm, tn;
        if (!tile_live(P, probs, t, &g, &tm, &tn)) continue;
        const int aslab = probs[g].a_slab, bslab = probs[g].b_slab;
        for (int pass = 0; ok && pass < 2; ++pass) {
          const int nd = pass ? ND : 4;
          ok = load_b_block(sB, fullB, emptyB, &tmB, &nbq, P.kb0, tn, bslab, nd);
          for (int u = 0; ok && u < P.nkb; ++u) {
            for (int p = 0; p < nd; ++p) {
              const int s = na % ASTAGES;
              if ((na >= ASTAGES && !mbar_wait(&emptyA[s], ((uint32_t)(na / ASTAGES) & 1u) ^ 1u)) ||
                  *(volatile int*)failed) {
                ok = false;
                break;
              }
              mbar_expect_tx(&fullA[s], A_BYTES);
              tma_load_3d(sA + s * A_BYTES, &tmA, &fullA[s], (P.kb0 + u) * BK, tm * BM, aslab * ND + p);
              ++na;
              // the next K block's B goes out early: its buffer was freed with block u - 1
              if (p == 1 && u + 1 < P.nkb &&
                  !load_b_block(sB, fullB, emptyB, &tmB, &nbq, P.kb0 + u + 1, tn, bslab, nd)) {
                ok = false;
                break;
              }
            }
          }
        }
      }
      if (!ok) atomicExch(failed, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer.  Pass 0: A digit p (0-3) times B digits
      // 0..3-p, into TMEM columns 64 p .. 255 (groups p..3).  Pass 1: A digit
      // p < 4 times B digits 4-p..7-p into columns 256-511 (groups 4-7), A
      // digit p >= 4 times B digits 0..7-p into columns 64 p .. 511.  Every
      // pair with p + q = g lands in group g's 64 columns.
      int na = 0, nbq = 0, it = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < total_tiles; t += gridDim.x) {
        int g, tm, tn;
        if (!tile_live(P, probs, t, &g, &tm, &tn)) continue;
        for (int pass = 0; ok && pass < 2; ++pass) {
          const int nd = pass ? ND : 4;
          // the epilogue has read this half of the previous tile's accumulators out
          if (it > 0 && !mbar_wait(&tempty[pass], (uint32_t)(it - 1) & 1u)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int u = 0; ok && u < P.nkb; ++u) {
            const int sb = nbq & 1;
            if (!mbar_wait(&fullB[sb], (uint32_t)(nbq >> 1) & 1u)) {
              ok = false;
              break;
            }
            const uint32_t b0 = smem_u32(sB + sb * B_BYTES);
            for (int p = 0; p < nd; ++p) {
              const int s = na % ASTAGES;
              if (!mbar_wait(&fullA[s], (uint32_t)(na / ASTAGES) & 1u)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const uint32_t a0 = smem_u32(sA + s * A_BYTES);
              int col, q0, nq;
              if (pass == 0) {
                col = 64 * p, q0 = 0, nq = 4 - p;
              } else if (p < 4) {
                col = 256, q0 = 4 - p, nq = 4;
              } else {
                col = 64 * p, q0 = 0, nq = ND - p;
              }
              const uint32_t id = idesc(64 * nq);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                // the first MMAs of a pass (digit 0 of the first K block) start its four groups
                const uint32_t acc = (u > 0 || p > 0 || kk > 0) ? 1u : 0u;
                umma(tmem + col, sdesc(a0 + kk * 32), sdesc(b0 + q0 * BQ_BYTES + kk * 32), id, acc);
              }
              umma_commit(&emptyA[s]);
              ++na;
            }
            umma_commit(&emptyB[sb]);
            ++nbq;
          }
          umma_commit(&tfull[pass]);  // arrives when every MMA of this half has completed
        }
        ++it;
      }
      if (!ok) atomicExch(failed, 1);
    }
  } else {
    // ---------------- epilogue warps: warp w reads TMEM lanes 32 (w mod 4) ..
    // (one row of the tile per thread) and one quarter of the columns.  It
    // reads groups 0-3 once the first pass is done (while the second runs),
    // keeps their Horner pairs and hands that half back; then groups 4-7
    // once the second pass is done (while the next tile's first pass runs),
    // combines and rounds, hands the second half back, and reads Cin and
    // writes each row's 16 entries (128 contiguous bytes per thread) under
    // the next tile's MMAs.
    const int q = warp & 3, c0 = 16 * ((warp - 2) >> 2);
    const bool neg_alpha = P.alpha < 0.0;  // alpha is +-1 and beta 0 or 1 (checked at launch)
    const bool use_cin = P.beta != 0.0;
    const bool small_k = P.nkb <= 2;  // K <= 128: every group sum within 2^22
    int it = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
      int g, tm, tn;
      if (!tile_live(P, probs, t, &g, &tm, &tn)) continue;
      const Problem pr = probs[g];
      const int grow = tm * BM + q * 32 + lane;
      const int col0 = tn * BN + c0;
      const int ei = P.ea[(int64_t)pr.a_slab * P.ea_rows + grow];
      const int fcol = P.eb[(int64_t)pr.b_slab * P.eb_rows + col0 + (lane & 15)];  // lane % 16 = column
      const bool row_ok = grow < pr.m;
      const bool row_cin = use_cin && pr.cin && row_ok && (grow < pr.nocin_r0 || grow >= pr.nocin_r1);
      const double* crow = row_cin ? pr.cin + (int64_t)grow * pr.ldcin + col0 : nullptr;
      if (row_cin && col0 < pr.n) {
        // the row's 16 addends (one or two 128-byte lines) into L2 while the
        // MMAs run; they are read after TMEM has been handed back
        asm volatile("prefetch.global.L2 [%0];" ::"l"(crow));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(crow + 15));
      }
      const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
      double* orow = pr.out + (int64_t)grow * pr.ldo;
      const bool vec_ok = ((reinterpret_cast<uintptr_t>(pr.out) | (uintptr_t)(pr.ldo * 8)) & 15u) == 0;
      const bool live = col0 < pr.n;  // else columns past this problem (narrow updates): nothing to read
      // Group sums within 2^22 in magnitude - always for K <= 128
      // (8 * 128 * 2^12), and for longer K whenever the warp's 16 sums of a
      // read are (checked) - become integers by an FP32 add: adding
      // 1.5 * 2^23 gives an FP32 in [2^23, 2^24] whose bit pattern less that
      // of 1.5 * 2^23 is the integer (at 2^24 the difference is still exactly
      // 2^22).  Otherwise (K up to 512: up to 2^24) a float-to-integer
      // conversion each.  A read: four groups (one half) of four columns, four
      // TMEM loads and a wait that names the loaded registers.
      uint32_t acc[4][4];
      auto read_half = [&](int half, int cq) -> bool {
#pragma unroll
        for (int gg = 0; gg < 4; ++gg) tmem_ld4_async(trow + 64 * (4 * half + gg) + c0 + cq, acc[gg]);
        tmem_wait_regs(acc);
        if (small_k) return true;
        float mx = 0.0f;
#pragma unroll
        for (int gg = 0; gg < 4; ++gg)
#pragma unroll
          for (int u = 0; u < 4; ++u) mx = fmaxf(mx, fabsf(__uint_as_float(acc[gg][u])));
        return __all_sync(0xffffffffu, mx <= 4194304.0f);
      };
      // the Horner pairs of one half: x0 = G_0 128 + G_1, x1 = G_2 128 + G_3
      // of its four groups, for column u of the read
      auto pairs = [&](bool fast, int u, int& x0, int& x1) {
        int a[4];
#pragma unroll
        for (int gg = 0; gg < 4; ++gg)
          a[gg] = fast ? __float_as_int(__uint_as_float(acc[gg][u]) + 12582912.0f) - 0x4B400000
                       : __float2int_rn(__uint_as_float(acc[gg][u]));
        x0 = a[0] * 128 + a[1];
        x1 = a[2] * 128 + a[3];
      };
      // ---- groups 0-3 (the first pass), kept as their Horner pairs
      bool ok = mbar_wait(&tfull[0], (uint32_t)it & 1u);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok || *(volatile int*)failed) {
        if (lane == 0 && P.err) atomicExch(P.err, 1);
        atomicExch(failed, 1);
        break;
      }
      // per column one 64-bit word: the first half's Horner pairs, then (in
      // the second half) the bits of the combined product
      unsigned long long hv[16];
      if (live) {
#pragma unroll
        for (int cq = 0; cq < 16; cq += 4) {
          const bool fast = read_half(0, cq);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            int x0, x1;
            pairs(fast, u, x0, x1);
            hv[cq + u] = ((unsigned long long)(uint32_t)x0 << 32) | (uint32_t)x1;
          }
        }
      }
      // this half has been read: the MMA warp may start the next tile's first pass
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[0]);
      // ---- groups 4-7 (the second pass), combined with the first half
      ok = mbar_wait(&tfull[1], (uint32_t)it & 1u);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok || *(volatile int*)failed) {
        if (lane == 0 && P.err) atomicExch(P.err, 1);
        atomicExch(failed, 1);
        break;
      }
      if (!live) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[1]);
      } else {
        // The combined products stay in registers; TMEM is released as soon
        // as the last columns are read, so the Schur update's add and the
        // stores run under the next tile's MMAs.
#pragma unroll
        for (int cq = 0; cq < 16; cq += 4) {
          const bool fast = read_half(1, cq);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c = cq + u;
            const int fj = __shfl_sync(0xffffffffu, fcol, c);
            int l0, l1;
            pairs(fast, u, l0, l1);
            const double v = (ei >= kNonFinite || fj >= kNonFinite)
                                 ? __longlong_as_double(0x7FF8000000000000LL)
                                 : combine((int)(hv[c] >> 32), (int)(uint32_t)hv[c], l0, l1, ei + fj - 61, neg_alpha);
            hv[c] = (unsigned long long)__double_as_longlong(v);
          }
        }
        // every accumulator of this tile has been read: the MMA warp may
        // start the next tile's second pass
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[1]);
        // the addends (from L2), the one FP64 instruction per entry - the
        // Schur update's add - and the stores: two columns per 16-byte access
        // where both are used (col is even; rows start on 16 bytes when the
        // base and leading dimension allow)
        double cpre[16];
        if (row_cin && col0 + 16 <= pr.n && ((reinterpret_cast<uintptr_t>(crow) & 15u) == 0)) {
#pragma unroll
          for (int c = 0; c < 16; c += 2) {
            const double2 t = *reinterpret_cast<const double2*>(crow + c);
            cpre[c] = t.x;
            cpre[c + 1] = t.y;
          }
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c) cpre[c] = (row_cin && col0 + c < pr.n) ? crow[c] : 0.0;
        }
#pragma unroll
        for (int cq = 0; cq < 16; cq += 2) {
          const int col = col0 + cq;
          const double v0 = cpre[cq] + __longlong_as_double((long long)hv[cq]),
                       v1 = cpre[cq + 1] + __longlong_as_double((long long)hv[cq + 1]);
          const bool w0 = row_ok && col < pr.n && (col < pr.skip_c0 || col >= pr.skip_c1);
          const bool w1 = row_ok && col + 1 < pr.n && (col + 1 < pr.skip_c0 || col + 1 >= pr.skip_c1);
          if (w0 && w1 && vec_ok) {
            *reinterpret_cast<double2*>(orow + col) = make_double2(v0, v1);
          } else {
            if (w0) orow[col] = v0;
            if (w1) orow[col + 1] = v1;
          }
        }
      }
      ++it;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// One CTA per rpc slab rows (64 for K <= 64, down to 8 for K >= 512: about
// 33 KB staged either way).  The source rows (or columns, transposed) are
// staged in shared memory up to 512 entries of K at a time: a slab of K <= 512
// is read from global memory once, all its loads in flight together; longer
// K takes two passes over chunks.  Pass 1 finds each row's largest magnitude
// (the bit patterns of |x| order like the values; Inf and NaN sort above every
// finite value), pass 2 writes the digits, four BF16 per lane and digit
// (256 contiguous bytes per warp instruction; two for chunks of 64 entries).
__global__ void __launch_bounds__(256, 4) oz_pack_kernel(const PackSet s0, const PackSet s1, int kpad, int rpc) {
  extern __shared__ double S[];  // [rpc][kc + 1]
  __shared__ int sE[PMAXR];
  __shared__ unsigned smx[PMAXR];  // running row maxima (high words of the bit patterns)
  // grid rows [0, s0.count) pack the slabs of the first set, the others those
  // of the second (two operands of one product in one launch)
  const bool second = (int)blockIdx.y >= s0.count;
  const PackSet ps = second ? s1 : s0;
  const int rows_pad = ps.rows_pad;
  __nv_bfloat16* __restrict__ dst = ps.dst;
  int* __restrict__ exps = ps.exps;
  const PackDesc d = ps.descs[second ? (int)blockIdx.y - s0.count : (int)blockIdx.y];
  const int r0 = blockIdx.x * rpc;
  if (r0 >= rows_pad) return;  // the grid covers the set with more slab rows
  const int rw = rpc / 8;  // rows per warp
  const int R = d.transpose ? d.cols : d.rows, KD = d.transpose ? d.rows : d.cols;
  // slab rows past the last 128-row tile that holds a source row are never
  // read (a product reads only the tiles of its problem's extent): leave them
  if (r0 >= (R + 127) / 128 * 128) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kc = kpad < PKC ? kpad : PKC;  // staged chunk of K
  const int lds = kc + 1;
  const int chunks = (kpad + kc - 1) / kc;
  // Stages entries [k0, k0 + kw) of the CTA's rows with asynchronous copies
  // (every copy of the stage in flight at once, none through registers);
  // entries past the source are zero-filled.
  auto load_chunk = [&](int k0) {
    const int kw = min(kc, kpad - k0);
    if (!d.transpose) {
      // thread (row group, column): for kw < 256 several rows go out at once
      const int tk = kw < 256 ? kw : 256;  // threads per row
      const int rg = tid / tk, kk0 = tid - rg * tk, rstep = 256 / tk;
      if (rg < rstep) {
        for (int rr = rg; rr < rpc; rr += rstep) {
          const int r = r0 + rr;
          for (int kk = kk0; kk < kw; kk += tk) {
            const int k = k0 + kk;
            const bool ok = r < R && k < KD;
            cp_async8(&S[rr * lds + kk], ok ? d.src + (int64_t)r * d.ld + k : d.src, ok);
          }
        }
      }
    } else {
      const int rr = tid & (rpc - 1);
      const int r = r0 + rr;
      for (int kk = tid / rpc; kk < kw; kk += 256 / rpc) {
        const int k = k0 + kk;
        const bool ok = r < R && k < KD;
        cp_async8(&S[rr * lds + kk], ok ? d.src + (int64_t)k * d.ld + r : d.src, ok);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  };
  // ---- pass 1: largest magnitude of each row (warp w: rows w rw .. w rw + rw - 1)
  for (int c = 0; c < chunks; ++c) {
    const int k0 = c * kc, kw = min(kc, kpad - k0);
    if (r0 >= R) break;
    if (c > 0) __syncthreads();
    load_chunk(k0);
    __syncthreads();
    // the exponent of the largest magnitude is in the high words alone (a row
    // whose high words are all zero holds zeros and subnormals, whose digits
    // are zero whatever E is)
    for (int h = 0; h < rw; ++h) {
      const int rr = warp * rw + h;
      const double* row = S + rr * lds;
      unsigned mx = 0;
      for (int kk = lane; kk < kw; kk += 32) {
        const unsigned hi = (unsigned)__double2hiint(row[kk]) & 0x7FFFFFFFu;
        mx = hi > mx ? hi : mx;
      }
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) smx[rr] = (c > 0 && smx[rr] > mx) ? smx[rr] : mx;
    }
  }
  __syncthreads();
  for (int rr = tid; rr < rpc; rr += 256) {
    const unsigned m = r0 < R ? smx[rr] : 0u;
    const int ex = (int)(m >> 20);
    // 2^E > max|x|: E = ex - 1022 for a normal maximum
    const int E = m == 0 ? 0 : (ex == 0x7ff ? kNonFinite : (ex == 0 ? -1022 : ex - 1022));
    sE[rr] = E;
    exps[(int64_t)d.slab * rows_pad + r0 + rr] = E;
  }
  // ---- pass 2: digits (a single chunk is still staged and is not read again)
  for (int c = 0; c < chunks; ++c) {
    const int k0 = c * kc, kw = min(kc, kpad - k0);
    __syncthreads();
    if (chunks > 1 || r0 >= R) {
      load_chunk(k0);
      __syncthreads();
    }
#pragma unroll 2
    for (int h = 0; h < rw; ++h) {
      const int rr = warp * rw + h;
      const int E = sE[rr];
      const double* row = S + rr * lds;
      __nv_bfloat16* out = dst + ((int64_t)d.slab * ND * rows_pad + r0 + rr) * kpad + k0;
      // four entries per lane, one 8-byte store per digit, when the chunk is
      // a multiple of 128 entries (the slab rows start on 128 bytes); else two
      // entries per lane (kw is a multiple of 64), so that no lane idles
      if (kw % 128) {
#pragma unroll 1
        for (int kk = 2 * lane; kk < kw; kk += 64) {
          int d0[ND], d1[ND];
          digits8(row[kk], E, d0);
          digits8(row[kk + 1], E, d1);
#pragma unroll
          for (int p = 0; p < ND; ++p)
            *(__nv_bfloat162*)&out[(int64_t)p * rows_pad * kpad + kk] = digit_pair(d0[p], d1[p]);
        }
        continue;
      }
#pragma unroll 1
      for (int kk = 4 * lane; kk < kw; kk += 128) {
        int d0[ND], d1[ND], d2[ND], d3[ND];
        digits8(row[kk], E, d0);
        digits8(row[kk + 1], E, d1);
        digits8(row[kk + 2], E, d2);
        digits8(row[kk + 3], E, d3);
#pragma unroll
        for (int p = 0; p < ND; ++p) {
          const __nv_bfloat162 lo = digit_pair(d0[p], d1[p]), hi = digit_pair(d2[p], d3[p]);
          uint2 v;
          v.x = *reinterpret_cast<const uint32_t*>(&lo);
          v.y = *reinterpret_cast<const uint32_t*>(&hi);
          *reinterpret_cast<uint2*>(&out[(int64_t)p * rows_pad * kpad + kk]) = v;
        }
      }
    }
  }
}

}  // namespace

unsigned long long g_stall_ns = 0;

void set_debug_stall(unsigned long long ns) { g_stall_ns = ns; }

int tile_m() { return BM; }
int tile_n() { return BN; }
int tile_k() { return BK; }
int pack_rows() { return PR; }
size_t smem_bytes() { return 2 * B_BYTES + ASTAGES * A_BYTES + 1024 + 256; }

cudaError_t launch_pack2(const PackSet& a, const PackSet& b, int kpad, cudaStream_t s) {
  const int count = (a.count > 0 ? a.count : 0) + (b.count > 0 ? b.count : 0);
  if (count <= 0) return cudaSuccess;
  for (const PackSet* p : {&a, &b})
    if (p->count > 0 && (p->rows_pad % PR || ((uintptr_t)p->dst & 3))) return cudaErrorInvalidValue;
  if (kpad % BK) return cudaErrorInvalidValue;
  {
    // the largest stage: 64 rows x 129 or 16 rows x 513 entries, about 66 KB
    cudaError_t e = once_per_device((const void*)oz_pack_kernel, [] {
      return cudaFuncSetAttribute(oz_pack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPackSmemMax);
    });
    if (e != cudaSuccess) return e;
  }
  const PackSet s0 = a.count > 0 ? a : b;
  PackSet s1 = a.count > 0 ? b : PackSet{};
  if (s1.count < 0) s1.count = 0;
  if (s0.count + s1.count > 65535 && s1.count > 0) {
    // beyond the grid's y extent together: one launch each
    cudaError_t e = launch_pack2(s0, PackSet{}, kpad, s);
    return e != cudaSuccess ? e : launch_pack2(s1, PackSet{}, kpad, s);
  }
  const int kc = kpad < PKC ? kpad : PKC;
  // rows per CTA: about 33 KB of staged entries, 8..64 rows (rows_pad is a
  // multiple of 64), so that four CTAs share an SM
  int rpc = (PR / 2) * (PKC / kc);
  rpc = rpc > PMAXR ? PMAXR : rpc;
  if (s0.rows_pad % rpc || (s1.count > 0 && s1.rows_pad % rpc)) rpc = PR;
  if ((size_t)rpc * (kc + 1) * sizeof(double) > (size_t)kPackSmemMax) return cudaErrorInvalidValue;
  const int rows = s1.count > 0 && s1.rows_pad > s0.rows_pad ? s1.rows_pad : s0.rows_pad;
  dim3 grid(rows / rpc, s0.count + s1.count);
  oz_pack_kernel<<<grid, 256, rpc * (kc + 1) * sizeof(double), s>>>(s0, s1, kpad, rpc);
  return cudaGetLastError();
}

cudaError_t launch_pack(const PackDesc* d_descs, int count, int rows_pad, int kpad, __nv_bfloat16* dst, int* exps,
                        cudaStream_t s) {
  return launch_pack2(PackSet{d_descs, count, rows_pad, dst, exps}, PackSet{}, kpad, s);
}

cudaError_t launch_gemm(const __nv_bfloat16* apk, int a_slabs, int a_rows_pad, const __nv_bfloat16* bpk, int b_slabs,
                        int b_rows_pad, const Params& P, const Problem* d_probs, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (P.kpad % BK || a_rows_pad % BM || b_rows_pad % BN || P.tiles_m * BM > a_rows_pad ||
      P.tiles_n * BN > b_rows_pad || P.nkb < 1 || P.nkb > kMaxKBlocks || P.kb0 < 0 ||
      (P.kb0 + P.nkb) * BK > P.kpad || P.ea_rows != a_rows_pad || P.eb_rows != b_rows_pad ||
      (P.alpha != 1.0 && P.alpha != -1.0) || (P.beta != 0.0 && P.beta != 1.0))
    return cudaErrorInvalidValue;
  if (((uintptr_t)apk | (uintptr_t)bpk) & 15) return cudaErrorInvalidValue;
  CUtensorMap ta, tb;
  if (!make_map(&ta, apk, P.kpad, a_rows_pad, a_slabs * ND, BM, BK, 1)) return cudaErrorInvalidValue;
  if (!make_map(&tb, bpk, P.kpad, b_rows_pad, b_slabs * ND, BN, BK, 4)) return cudaErrorInvalidValue;
  const size_t sm = smem_bytes();
  {
    cudaError_t e = once_per_device((const void*)oz_gemm_kernel, [sm] {
      return cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    });
    if (e != cudaSuccess) return e;
  }
  Params Q = P;
  Q.stall_ns = g_stall_ns;
  const int sms = sm_count();
  const int total = count * P.tiles_m * P.tiles_n;
  int grid = total < sms ? total : sms;
  if (P.coprime_grid) {
    auto gcd = [](int a, int b) {
      while (b) {
        const int t = a % b;
        a = b;
        b = t;
      }
      return a;
    };
    while (grid > 1 && gcd(grid, P.tiles_n) != 1) --grid;
  }
  oz_gemm_kernel<<<grid, THREADS, sm, s>>>(ta, tb, Q, d_probs, total);
  return cudaGetLastError();
}

}  // namespace oz
}  // namespace mbinv
