// Test hooks of the tensor-core products (not part of the public header): run
// the grouped tcgen05 GEMMs on plain row-major inputs so that the tests can
// check them against a plain product without going through the recursion.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <limits>
#include <vector>

#include "exec.h"
#include "mbinv_internal.h"
#include "ozaki.h"
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

// C[g] = beta * Cin[g] + alpha * A[g] B[g] for count row-major FP64 problems
// (A m x k, B k x n, Cin and C m x n; Cin may be null) through the digit-split
// FP64 product, in K chunks of at most 512 as the executor runs it.
extern "C" int mbinv_debug_oz_gemm(const double* A, const double* B, const double* Cin, double* C, int m, int n,
                                   int k, int count, double alpha, double beta, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int TM = oz::tile_m(), TN = oz::tile_n(), KT = oz::tile_k(), ND = oz::kDigits;
  const int mpad = (m + TM - 1) / TM * TM, npad = (n + TN - 1) / TN * TN, kpad = (k + KT - 1) / KT * KT;
  __nv_bfloat16 *apk = nullptr, *bpk = nullptr;
  int *ea = nullptr, *eb = nullptr, *derr = nullptr;
  oz::PackDesc* dd = nullptr;
  oz::Problem* dp = nullptr;
  int rc = 0;
  if (cudaMalloc(&apk, (size_t)count * ND * mpad * kpad * 2) || cudaMalloc(&bpk, (size_t)count * ND * npad * kpad * 2) ||
      cudaMalloc(&ea, sizeof(int) * count * mpad) || cudaMalloc(&eb, sizeof(int) * count * npad) ||
      cudaMalloc(&dd, sizeof(oz::PackDesc) * 2 * count) || cudaMalloc(&dp, sizeof(oz::Problem) * 2 * count) ||
      cudaMalloc(&derr, sizeof(int)))
    rc = 1;
  if (!rc) {
    std::vector<oz::PackDesc> pd(2 * count);
    std::vector<oz::Problem> pr(2 * count);
    for (int g = 0; g < count; ++g) {
      pd[g] = oz::PackDesc{A + (size_t)g * m * k, k, m, k, 0, g};
      pd[count + g] = oz::PackDesc{B + (size_t)g * k * n, n, k, n, 1, g};  // slab row = column of B
      double* out = C + (size_t)g * m * n;
      pr[g] = oz::Problem{g, g, Cin ? Cin + (size_t)g * m * n : nullptr, n, out, n, m, n, 0, 0, 0, 0};
      pr[count + g] = oz::Problem{g, g, out, n, out, n, m, n, 0, 0, 0, 0};  // later K chunks accumulate into C
    }
    cudaMemcpyAsync(dd, pd.data(), sizeof(oz::PackDesc) * 2 * count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dp, pr.data(), sizeof(oz::Problem) * 2 * count, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(derr, 0, sizeof(int), s);
    if (oz::launch_pack(dd, count, mpad, kpad, apk, ea, s) != cudaSuccess) rc = 2;
    if (!rc && oz::launch_pack(dd + count, count, npad, kpad, bpk, eb, s) != cudaSuccess) rc = 3;
    oz::Params P{};
    P.kpad = kpad;
    P.tiles_m = mpad / TM;
    P.tiles_n = npad / TN;
    P.alpha = alpha;
    P.ea = ea;
    P.eb = eb;
    P.ea_rows = mpad;
    P.eb_rows = npad;
    P.err = derr;
    const int nkb = kpad / KT;
    for (int kb0 = 0; !rc && kb0 < nkb; kb0 += oz::kMaxKBlocks) {
      P.kb0 = kb0;
      P.nkb = nkb - kb0 < oz::kMaxKBlocks ? nkb - kb0 : oz::kMaxKBlocks;
      P.beta = kb0 == 0 ? beta : 1.0;
      if (oz::launch_gemm(apk, count, mpad, bpk, count, npad, P, dp + (kb0 == 0 ? 0 : count), count, s) !=
          cudaSuccess)
        rc = 4;
    }
    int herr = 0;
    if (!rc && cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = 5;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = 6;
    if (!rc && herr) rc = 7;
  }
  cudaFree(apk);
  cudaFree(bpk);
  cudaFree(ea);
  cudaFree(eb);
  cudaFree(dd);
  cudaFree(dp);
  cudaFree(derr);
  return rc;
}

// Host-only hook of the planner (no CUDA call): for block (i, j) of a k x k
// grid, out[0] distinct frames, out[1] order-2 (leaf) frames, out[2] inverses
// of the schedule (distinct pivots plus the root), out[3] peak value slots,
// out[4] product work and out[5] inverse work, both in units of b^3 (2 per
// b x b x b product, 2 per b x b inverse).  0, or -1 for invalid arguments.
extern "C" int mbinv_debug_plan(int k, int i, int j, int pad_last, double* out) {
  if (k < 1 || i < 0 || j < 0 || i >= k || j >= k || !out) return -1;
  try {
    const Plan P = build_plan(k, i, j, pad_last != 0);
    const Schedule S = build_schedule(P, 0);
    out[0] = (double)S.frames;
    out[1] = (double)P.leaves;
    out[2] = (double)S.inversions;
    out[3] = (double)S.nslots;
    out[4] = S.gemm_flops_units;
    out[5] = S.inv_units;
  } catch (...) {
    return -1;
  }
  return 0;
}

// Host-only hook of the merged planner (no CUDA call): the requests ij[2t],
// ij[2t+1] (t < count) of a k x k grid planned together.  out[0] frames
// evaluated, out[1] frames of the requests run one by one, out[2] inverses,
// out[3] peak value slots, out[4] product work and out[5] inverse work in
// units of b^3, out[6] leaves.  0, or -1 for invalid arguments.
extern "C" int mbinv_debug_plan_group(int k, int count, const int* ij, int pad_last, double* out) {
  if (k < 2 || count < 1 || !ij || !out) return -1;
  try {
    std::vector<std::pair<int, int>> reqs;
    for (int t = 0; t < count; ++t) {
      if (ij[2 * t] < 0 || ij[2 * t + 1] < 0 || ij[2 * t] >= k || ij[2 * t + 1] >= k) return -1;
      reqs.emplace_back(ij[2 * t], ij[2 * t + 1]);
    }
    const Plan P = build_plan(k, reqs, pad_last != 0);
    const Schedule S = build_schedule(P, 0);
    out[0] = (double)S.frames;
    out[1] = (double)S.request_frames;
    out[2] = (double)S.inversions;
    out[3] = (double)S.nslots;
    out[4] = S.gemm_flops_units;
    out[5] = S.inv_units;
    out[6] = (double)P.leaves;
  } catch (...) {
    return -1;
  }
  return 0;
}

// Host-only hook (no CUDA call): builds the schedule of the requests ij (count
// pairs) on a k x k grid and runs it on scalars, b = 1: M is k x k row-major,
// an inverse is 1/x, a product alpha A B + beta Cin, a copy moves a value.
// mode 0: level by level; mode 1: bounded, in `slots` slots, M blocks read
// from "host memory" when host_m; mode 2: the principal-Schur variant (one
// request).  outs[t] receives request t's result;
// stats: steps, peak slots, host spill slots, loads, spills, inversions,
// product units (b^3).  0; -1 for invalid arguments; -2 when the schedule
// cannot be built in that many slots; -3 when a value is read before it is
// written.
extern "C" int mbinv_debug_run_schedule_scalar(int k, int count, const int* ij, int mode, int slots, int host_m,
                                               const double* M, double* outs, double* stats) {
  if (k < 2 || count < 1 || !ij || !M || !outs || !stats) return -1;
  try {
    std::vector<std::pair<int, int>> reqs;
    for (int t = 0; t < count; ++t) {
      if (ij[2 * t] < 0 || ij[2 * t + 1] < 0 || ij[2 * t] >= k || ij[2 * t + 1] >= k) return -1;
      reqs.emplace_back(ij[2 * t], ij[2 * t + 1]);
    }
    const Plan P = build_plan(k, reqs, false);
    Schedule S;
    if (mode == 0) S = build_schedule(P, 0);
    else if (mode == 2) {
      if (count != 1) return -1;
      S = build_psc_schedule(k, ij[0], ij[1]);
    } else if (!build_bounded_schedule(P, slots, host_m != 0, &S)) return -2;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    std::vector<double> sl((size_t)std::max(1, S.nslots), nan), sp((size_t)std::max(1, S.nspill), nan);
    std::vector<char> wsl(sl.size(), 0), wsp(sp.size(), 0);
    for (int t = 0; t < count; ++t) outs[t] = nan;
    bool bad = false;
    auto rd = [&](const Ref& r) -> double {
      switch (r.kind) {
        case Ref::MBLK:
        case Ref::HOSTM: return M[r.r * k + r.c];
        case Ref::SLOT: if (!wsl.at(r.slot)) bad = true; return sl.at(r.slot);
        case Ref::SPILL: if (!wsp.at(r.slot)) bad = true; return sp.at(r.slot);
        default: bad = true; return nan;
      }
    };
    auto wr = [&](const Ref& r, double v) {
      if (r.kind == Ref::SLOT) { sl.at(r.slot) = v; wsl.at(r.slot) = 1; }
      else if (r.kind == Ref::SPILL) { sp.at(r.slot) = v; wsp.at(r.slot) = 1; }
      else if (r.kind == Ref::OUT) outs[r.slot] = v;
      else bad = true;
    };
    for (const Step& st : S.steps) {
      for (const CopyOp& c : st.copy) wr(c.dst, rd(c.src));
      for (const InvOp& io : st.inv) wr(io.dst, 1.0 / rd(io.src));
      for (const GemmOp& g : st.gemm) {
        const double p = rd(g.A) * rd(g.B);
        double v = g.alpha < 0 ? -p : p;
        if (g.Cin.kind != Ref::NONE && g.beta != 0.0) v = g.alpha < 0 ? rd(g.Cin) - p : rd(g.Cin) + p;
        wr(g.C, v);
      }
    }
    if (bad) return -3;
    stats[0] = (double)S.steps.size();
    stats[1] = (double)S.nslots;
    stats[2] = (double)S.nspill;
    stats[3] = (double)S.loads;
    stats[4] = (double)S.spills;
    stats[5] = (double)S.inversions;
    stats[6] = S.gemm_flops_units;
  } catch (...) {
    return -1;
  }
  return 0;
}

// Test hooks of the failure paths (no fault is made on the GPU):
// every later digit-product launch first waits `ns` nanoseconds on a barrier
// nothing arrives at and returns having raised its error word (0 = off); the
// next `n` device allocations of the library fail as if the GPU were out of
// memory.
extern "C" void mbinv_debug_set_stall_ns(unsigned long long ns) { oz::set_debug_stall(ns); }
extern "C" void mbinv_debug_fail_allocations(int n) { injected_alloc_failures() = n > 0 ? n : 0; }

namespace {

// Descriptors of count independent products out_g = Cin_g - A_g B_g (n x n,
// row-major, consecutive in memory).
__global__ void products_setup_kernel(const double* A, const double* B, const double* Cin, double* C, int n,
                                      int count, oz::PackDesc* pd, oz::Problem* pr) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const size_t off = (size_t)g * n * n;
  pd[g] = oz::PackDesc{A + off, n, n, n, 0, g};
  pd[count + g] = oz::PackDesc{B + off, n, n, n, 1, g};  // slab row = column of B
  pr[g] = oz::Problem{g, g, Cin + off, n, C + off, n, n, n, 0, 0, 0, 0};
}

}  // namespace

// Bytes of workspace mbinv_debug_oz_products needs for count products of
// order n (n <= 512).
extern "C" size_t mbinv_debug_oz_products_bytes(int n, int count) {
  const int TM = oz::tile_m(), TN = oz::tile_n(), KT = oz::tile_k();
  const size_t mpad = (n + TM - 1) / TM * TM, npad = (n + TN - 1) / TN * TN, kpad = (n + KT - 1) / KT * KT;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return al(count * oz::kDigits * mpad * kpad * 2) + al(count * oz::kDigits * npad * kpad * 2) +
         al(count * mpad * 4) + al(count * npad * 4) + al(2 * count * sizeof(oz::PackDesc)) +
         al(count * sizeof(oz::Problem)) + al(sizeof(int));
}

// count products out_g = Cin_g - A_g B_g of order n <= 512 (one K chunk) on
// the FP64_TC digit-product kernels, in caller-given device workspace, with
// no allocation and no synchronisation: a setup kernel, two packs and one
// grouped product on the stream (the Schur products' kernels, timed alone).
// pack = 0 launches the product alone, on the digits an earlier call with
// the same operands and workspace left there.  0, or nonzero for invalid
// arguments or a launch error.
extern "C" int mbinv_debug_oz_products(const double* A, const double* B, const double* Cin, double* C, int n,
                                       int count, void* ws, size_t ws_bytes, int pack, void* stream) {
  if (n < 1 || n > 512 || count < 1 || !A || !B || !Cin || !C || !ws ||
      ws_bytes < mbinv_debug_oz_products_bytes(n, count))
    return 1;
  cudaStream_t s = (cudaStream_t)stream;
  const int TM = oz::tile_m(), TN = oz::tile_n(), KT = oz::tile_k();
  const int mpad = (n + TM - 1) / TM * TM, npad = (n + TN - 1) / TN * TN, kpad = (n + KT - 1) / KT * KT;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* p = (char*)ws;
  auto* apk = (__nv_bfloat16*)p;
  p += al((size_t)count * oz::kDigits * mpad * kpad * 2);
  auto* bpk = (__nv_bfloat16*)p;
  p += al((size_t)count * oz::kDigits * npad * kpad * 2);
  int* ea = (int*)p;
  p += al((size_t)count * mpad * 4);
  int* eb = (int*)p;
  p += al((size_t)count * npad * 4);
  auto* pd = (oz::PackDesc*)p;
  p += al(2 * (size_t)count * sizeof(oz::PackDesc));
  auto* pr = (oz::Problem*)p;
  p += al((size_t)count * sizeof(oz::Problem));
  int* derr = (int*)p;
  if (pack) {
    products_setup_kernel<<<(count + 127) / 128, 128, 0, s>>>(A, B, Cin, C, n, count, pd, pr);
    if (cudaGetLastError() != cudaSuccess) return 2;
    if (oz::launch_pack(pd, count, mpad, kpad, apk, ea, s) != cudaSuccess) return 3;
    if (oz::launch_pack(pd + count, count, npad, kpad, bpk, eb, s) != cudaSuccess) return 4;
  }
  oz::Params P{};
  P.kpad = kpad;
  P.kb0 = 0;
  P.nkb = kpad / KT;
  P.tiles_m = mpad / TM;
  P.tiles_n = npad / TN;
  P.alpha = -1.0;
  P.beta = 1.0;
  P.ea = ea;
  P.eb = eb;
  P.ea_rows = mpad;
  P.eb_rows = npad;
  P.err = derr;
  return oz::launch_gemm(apk, count, mpad, bpk, count, npad, P, pr, count, s) == cudaSuccess ? 0 : 5;
}
