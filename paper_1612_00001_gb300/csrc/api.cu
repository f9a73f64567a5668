// C ABI of libmbinv and the executor of the recursion's schedule.
//
// mbinv_block(i, j) plans the recursion for block (i, j) on the host (no
// arithmetic, Sec. 3.1), then runs it level by level on one CUDA stream
// (Sec. 3.2): per level one batched pivot inversion and two grouped Schur
// products, so that every frame of a level is in flight at once.  Values
// live in fixed-size b x b slots of one workspace; the planner decides which
// slot holds which value and frees a level's inputs as soon as the level is
// done, which bounds the workspace by the two widest adjacent levels.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <climits>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <stdexcept>
#include <vector>

#include "../../include/mbinv.h"
#include "mbinv_internal.h"
#include "tc_gemm.h"

using namespace mbinv;

#define CU(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      last_cuda_error() = e_;                   \
      return MBINV_ECUDA;                       \
    }                                           \
  } while (0)

namespace {

cudaError_t& last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// SplitMix64 (Steele, Lea and Flood 2014) as a counter-based generator:
// draw t of stream (seed, stream) = mix(mix(seed ^ mix(stream)) + (t+1) * golden).
__host__ __device__ inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Coupling block of the border: rows [0, n) x columns [n, n + l) get
// B'[r][q] (request (i, k-1)), or rows [n, n+l) x columns [0, n) get
// C'[q][c] = B'[c][q] (request (k-1, j)); B'[r][q] = uniform[-1,1) draw r*l+q.
template <typename T>
__global__ void border_kernel(T* g, int64_t ldg, int64_t n, int64_t l, uint64_t seed, int mode) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * l) return;
  const int64_t r = e / l, q = e % l;
  double v = 0.0;
  if (mode != 0) {
    const uint64_t base = sm64_mix(seed ^ sm64_mix(6ull));
    const uint64_t u = sm64_mix(base + (uint64_t)(e + 1) * 0x9E3779B97F4A7C15ull);
    v = 2.0 * ((double)(u >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
  }
  // top-right strip (coupling when mode == 1, zero otherwise)
  g[r * ldg + n + q] = (mode == 1) ? (T)v : (T)0;
  // bottom-left strip (coupling when mode == 2, zero otherwise)
  g[(n + q) * ldg + r] = (mode == 2) ? (T)v : (T)0;
}

// dst[r][c] = (TD) src[r][c]
template <typename TS, typename TD>
__global__ void convert_kernel(const TS* src, int64_t lds, TD* dst, int64_t ldd, int64_t rows, int64_t cols) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = e / cols, q = e % cols;
  dst[r * ldd + q] = (TD)src[r * lds + q];
}

// R[r][i0 + r] += 1 for r < b: E_i^T - X_i M from -X_i M.
__global__ void add_eye_kernel(double* R, int64_t ldr, int64_t i0, int64_t b) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < b) R[r * ldr + i0 + r] += 1.0;
}

// sum of squares of an m x n FP64 matrix into *acc (one atomic per warp)
__global__ void sumsq_kernel(const double* R, int64_t ldr, int64_t m, int64_t n, double* acc) {
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * n; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = R[(e / n) * ldr + e % n];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, need);
    if (e == cudaSuccess) bytes = need;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

struct HostBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMallocHost(&p, need);
    if (e == cudaSuccess) bytes = need;
    return e;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
  }
};

}  // namespace

struct mbinv_ctx {
  int64_t n = 0, k = 0, b = 0, npad = 0, l = 0;
  int dtype = F64;  // the caller's element type (M, outputs, G, dM)
  int mdt = F64;    // element type of the device copy of M the sweep reads
  mbinv_options opt{};
  cudaStream_t stream = nullptr;
  // device copy (or borrowed pointer) of M, or of the bordered matrix
  const void* dM = nullptr;
  int64_t ldm = 0;
  DevBuf own_M;
  int border_mode = -1;  // border strips currently written (-1: none yet)
  // workspace
  DevBuf slots, inv_work, inv_wrow, inv_perm, inv_amax, desc, status, outtmp, rowbuf, colbuf, resid;
  DevBuf apk, bpk, b2pk, tcerr;  // mixed path: packed BF16 operand slabs
  HostBuf hdesc, hstage;
  std::vector<cudaEvent_t> events;  // profiling: pairs around launches
  bool in_sweep = false;            // refinement: inner sweeps run unrefined
  size_t own_bytes = 0;  // peak of what this context holds on the device
  std::map<std::pair<int, int>, std::pair<Plan, Schedule>> plans;
};

namespace {

int work_type(const mbinv_ctx* c) { return c->opt.precision == MBINV_FP32 ? F32 : F64; }
int slot_type(const mbinv_ctx* c) { return c->opt.precision == MBINV_FP64 ? F64 : F32; }

size_t slot_bytes(const mbinv_ctx* c) {
  size_t s = (size_t)c->b * c->b * dtype_size(slot_type(c));
  return (s + 255) & ~(size_t)255;
}

size_t inv_scratch_bytes(const mbinv_ctx* c, int count) {
  const size_t ws = dtype_size(work_type(c));
  const size_t b = (size_t)c->b;
  const size_t nb = (size_t)inv_panel_width((int)b, work_type(c));
  return (size_t)count * (b * b * ws + 256 + nb * b * ws + 256 + b * 4 + 256 + 256);
}

// Total device bytes a schedule needs beyond M.
size_t schedule_bytes(const mbinv_ctx* c, const Schedule& S, int inv_chunk) {
  return (size_t)S.nslots * slot_bytes(c) + inv_scratch_bytes(c, inv_chunk) + 2 * slot_bytes(c) + (1 << 20);
}

mbinv_status ensure_workspace(mbinv_ctx* c, const Schedule& S, int inv_chunk) {
  const size_t sb = slot_bytes(c);
  CU(c->slots.ensure((size_t)S.nslots * sb));
  const size_t ws = dtype_size(work_type(c));
  const size_t b = (size_t)c->b;
  const size_t nb = (size_t)inv_panel_width((int)b, work_type(c));
  CU(c->inv_work.ensure((size_t)inv_chunk * ((b * b * ws + 255) & ~(size_t)255)));
  CU(c->inv_wrow.ensure((size_t)inv_chunk * ((nb * b * ws + 255) & ~(size_t)255)));
  CU(c->inv_perm.ensure((size_t)inv_chunk * ((b * 4 + 255) & ~(size_t)255)));
  CU(c->inv_amax.ensure((size_t)inv_chunk * 256));
  CU(c->outtmp.ensure((size_t)c->b * c->b * 8 + 256));
  CU(c->status.ensure(256));
  size_t total = c->slots.bytes + c->inv_work.bytes + c->inv_wrow.bytes + c->inv_perm.bytes + c->inv_amax.bytes +
                 c->outtmp.bytes + c->status.bytes + c->own_M.bytes + c->desc.bytes;
  c->own_bytes = std::max(c->own_bytes, total);
  return MBINV_OK;
}

// Chooses the Schur-temporary chunk and the inverse batch chunk so that the
// plan fits the cap; returns false when nothing fits.
bool fit_cap(const mbinv_ctx* c, const Plan& P, Schedule* S, int* inv_chunk) {
  const size_t cap = c->opt.device_cap_bytes;
  const size_t base = c->own_M.bytes;
  *S = build_schedule(P, 0);
  *inv_chunk = std::max(1, S->max_inv_batch);
  if (cap == 0) return true;
  for (int z : {0, 64, 16, 4, 1}) {
    Schedule T = build_schedule(P, z);
    for (int ic : {std::max(1, T.max_inv_batch), 64, 16, 4, 1}) {
      if (ic > std::max(1, T.max_inv_batch)) continue;
      if (base + schedule_bytes(c, T, ic) <= cap) {
        *S = T;
        *inv_chunk = ic;
        return true;
      }
    }
  }
  return false;
}

struct Exec {
  mbinv_ctx* c;
  const Schedule* S;
  void* out;  // device destination of the final inverse
  int64_t ldo;
  int out_dtype;
  int inv_chunk;
  int launches = 0;
  int gemm_launches = 0;
  double gemm_dev_s = 0, inv_dev_s = 0, pack_dev_s = 0;
};

cudaError_t ensure_events(mbinv_ctx* c, size_t n) {
  while (c->events.size() < n) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    c->events.push_back(e);
  }
  return cudaSuccess;
}

const void* resolve(const mbinv_ctx* c, const Ref& r, const Exec& X, int64_t* ld, int* dt) {
  switch (r.kind) {
    case Ref::MBLK: {
      *ld = c->ldm;
      *dt = c->mdt;
      const size_t es = dtype_size(c->mdt);
      return (const char*)c->dM + ((size_t)r.r * c->b * c->ldm + (size_t)r.c * c->b) * es;
    }
    case Ref::SLOT:
      *ld = c->b;
      *dt = slot_type(c);
      return (const char*)c->slots.p + (size_t)r.slot * slot_bytes(c);
    case Ref::OUT:
      *ld = X.ldo;
      *dt = X.out_dtype;
      return X.out;
    default:
      *ld = 0;
      *dt = -1;
      return nullptr;
  }
}

int combo_for(int adt, int bdt, int cdt) {
  if (adt == F64 && bdt == F64 && cdt == F64) return G_F64;
  if (adt == F32 && bdt == F32 && cdt == F32) return G_F32;
  if (adt == F32 && bdt == F32 && cdt == F64) return G_F32IN_F64;
  if (adt == F64 && bdt == F32 && cdt == F64) return G_F64F32_F64;
  return -1;
}

// Runs an FP64 / FP32 schedule (CUDA-core products).
mbinv_status run_schedule(Exec& X) {
  mbinv_ctx* c = X.c;
  const Schedule& S = *X.S;
  // descriptor arena: all steps' descriptors are written to pinned host memory
  // and copied in one transfer
  size_t need = 0;
  for (const Step& st : S.steps) {
    const size_t nchunks = st.kind == Step::INV ? (st.inv.size() + X.inv_chunk - 1) / X.inv_chunk : 1;
    need += (st.kind == Step::INV ? st.inv.size() * sizeof(InvDesc) : st.gemm.size() * sizeof(GemmDesc)) +
            256 * nchunks;
  }
  need += 256;  // status words at the end of the pinned buffer
  CU(c->desc.ensure(need));
  CU(c->hdesc.ensure(need));
  char* hbase = (char*)c->hdesc.p;
  char* dbase = (char*)c->desc.p;
  size_t off = 0;
  struct Launch {
    int kind;
    size_t off;
    int count;
    int combo;
    int tiles;
    int in_dt, out_dt;
  };
  std::vector<Launch> L;
  const size_t ws = dtype_size(work_type(c));
  const size_t b = (size_t)c->b;
  const size_t nb = (size_t)inv_panel_width((int)b, work_type(c));
  const size_t wstride = (b * b * ws + 255) & ~(size_t)255;
  const size_t rstride = (nb * b * ws + 255) & ~(size_t)255;
  const size_t pstride = (b * 4 + 255) & ~(size_t)255;
  int inv_tag = 0;
  for (const Step& st : S.steps) {
    if (st.kind == Step::INV) {
      for (size_t c0 = 0; c0 < st.inv.size(); c0 += X.inv_chunk) {
        const size_t c1 = std::min(st.inv.size(), c0 + (size_t)X.inv_chunk);
        InvDesc* hd = (InvDesc*)(hbase + off);
        int in_dt = -1, out_dt = -1;
        for (size_t t = c0; t < c1; ++t) {
          InvDesc d{};
          int64_t ld;
          d.src = resolve(c, st.inv[t].src, X, &ld, &in_dt);
          d.lds = ld;
          d.dst = (void*)resolve(c, st.inv[t].dst, X, &ld, &out_dt);
          d.ldd = ld;
          d.work = (char*)c->inv_work.p + (t - c0) * wstride;
          d.wrow = (char*)c->inv_wrow.p + (t - c0) * rstride;
          d.perm = (int*)((char*)c->inv_perm.p + (t - c0) * pstride);
          d.amax = (unsigned long long*)((char*)c->inv_amax.p + (t - c0) * 256);
          d.b = (int)b;
          d.tag = inv_tag++;
          hd[t - c0] = d;
        }
        L.push_back({0, off, (int)(c1 - c0), 0, 0, in_dt, out_dt});
        off += ((c1 - c0) * sizeof(InvDesc) + 255) & ~(size_t)255;
      }
    } else {
      if (st.gemm.empty()) continue;
      GemmDesc* hd = (GemmDesc*)(hbase + off);
      int combo = -1, tiles = 0;
      for (size_t t = 0; t < st.gemm.size(); ++t) {
        const GemmOp& g = st.gemm[t];
        GemmDesc d{};
        int adt, bdt, cdt, idt = -1;
        int64_t ld;
        d.A = resolve(c, g.A, X, &ld, &adt);
        d.lda = ld;
        d.B = resolve(c, g.B, X, &ld, &bdt);
        d.ldb = ld;
        d.C = (void*)resolve(c, g.C, X, &ld, &cdt);
        d.ldc = ld;
        if (g.Cin.kind != Ref::NONE) {
          d.Cin = resolve(c, g.Cin, X, &ld, &idt);
          d.ldcin = ld;
        }
        d.m = d.n = d.k = (int)b;
        d.alpha = g.alpha;
        d.beta = g.beta;
        const int cb = combo_for(adt, bdt, cdt);
        if (cb < 0 || (combo >= 0 && cb != combo) || (idt >= 0 && idt != cdt)) return MBINV_ENOTSUP;
        combo = cb;
        int bm, bn;
        gemm_tile_shape(combo, &bm, &bn);
        d.tiles_n = (d.n + bn - 1) / bn;
        d.tile_start = tiles;
        tiles += ((d.m + bm - 1) / bm) * d.tiles_n;
        hd[t] = d;
      }
      L.push_back({1, off, (int)st.gemm.size(), combo, tiles, 0, 0});
      off += (st.gemm.size() * sizeof(GemmDesc) + 255) & ~(size_t)255;
    }
  }
  CU(cudaMemcpyAsync(dbase, hbase, off, cudaMemcpyHostToDevice, c->stream));
  DevStatus* hst = (DevStatus*)(hbase + need - sizeof(DevStatus) * 2);
  hst[0] = DevStatus{0, INT_MAX};
  CU(cudaMemcpyAsync(c->status.p, &hst[0], sizeof(DevStatus), cudaMemcpyHostToDevice, c->stream));
  const bool prof = c->opt.profile != 0;
  if (prof) CU(ensure_events(c, 2 * L.size()));
  for (size_t q = 0; q < L.size(); ++q) {
    const Launch& l = L[q];
    if (prof) CU(cudaEventRecord(c->events[2 * q], c->stream));
    if (l.kind == 0) {
      CU(run_inverse_batch(l.in_dt, l.out_dt, work_type(c), (const InvDesc*)(dbase + l.off), l.count, (int)b,
                           (DevStatus*)c->status.p, c->stream, &X.launches));
    } else {
      CU(launch_gemm_grouped(l.combo, (const GemmDesc*)(dbase + l.off), l.count, l.tiles, c->stream));
      ++X.launches;
      ++X.gemm_launches;
    }
    if (prof) CU(cudaEventRecord(c->events[2 * q + 1], c->stream));
  }
  CU(cudaMemcpyAsync(&hst[1], c->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  const DevStatus st = hst[1];
  if (prof) {
    for (size_t q = 0; q < L.size(); ++q) {
      float ms = 0;
      CU(cudaEventElapsedTime(&ms, c->events[2 * q], c->events[2 * q + 1]));
      (L[q].kind == 0 ? X.inv_dev_s : X.gemm_dev_s) += ms * 1e-3;
    }
  }
  if (st.singular) return MBINV_ESINGULAR;
  return MBINV_OK;
}

// Runs a schedule on the mixed path: pivot inverses as in run_schedule (FP64
// Gauss-Jordan, FP32 results), every Schur product on the tensor cores.  A
// pair of GEMM steps Z = P^-1 R, X = K - L Z becomes: pack the distinct P^-1
// (row-major slices) and every R (transposed slices), tcgen05 product with the
// slices of Z^T written straight into the B operand of the second product,
// pack the distinct L, tcgen05 product with the fused subtraction from K.
mbinv_status run_schedule_mixed(Exec& X) {
  mbinv_ctx* c = X.c;
  const Schedule& S = *X.S;
  const int b = (int)c->b;
  const int T = tc::tile_rows(), KT = tc::tile_k();
  const int rpad = (b + T - 1) / T * T, kpad = (b + KT - 1) / KT * KT;
  const int NS = c->opt.bf16_slices;
  const size_t slab = (size_t)NS * rpad * kpad;  // bf16 elements per packed operand
  // pass 1: sizes
  size_t maxA = 1, maxB = 1, need = 256;
  for (const Step& st : S.steps) {
    if (st.kind == Step::INV) {
      const size_t nchunks = (st.inv.size() + X.inv_chunk - 1) / X.inv_chunk;
      need += st.inv.size() * sizeof(InvDesc) + 256 * nchunks;
    } else {
      std::map<std::pair<int, int>, int> da;
      for (const GemmOp& g : st.gemm) da[{g.A.kind == Ref::SLOT ? g.A.slot : -1 - g.A.r, g.A.c}] = 0;
      maxA = std::max(maxA, da.size());
      maxB = std::max(maxB, st.gemm.size());
      need += (da.size() + st.gemm.size()) * sizeof(tc::PackDesc) + st.gemm.size() * sizeof(tc::TcProblem) + 768;
    }
  }
  CU(c->apk.ensure(maxA * slab * 2));
  CU(c->bpk.ensure(maxB * slab * 2));
  CU(c->b2pk.ensure(maxB * slab * 2));
  CU(c->tcerr.ensure(256));
  CU(c->desc.ensure(need));
  CU(c->hdesc.ensure(need));
  char* hbase = (char*)c->hdesc.p;
  char* dbase = (char*)c->desc.p;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  struct Launch {
    int kind;  // 0 inverse, 1 pack A, 2 pack B, 3 tc gemm
    size_t off;
    int count;
    int in_dt, out_dt;
    int nA;  // tc gemm: slabs of A
    int mode;
    __nv_bfloat16 *adst, *bsrc;
  };
  std::vector<Launch> L;
  const size_t ws = 8;
  const size_t nb = (size_t)inv_panel_width(b, F64);
  const size_t wstride = ((size_t)b * b * ws + 255) & ~(size_t)255;
  const size_t rstride = (nb * b * ws + 255) & ~(size_t)255;
  const size_t pstride = ((size_t)b * 4 + 255) & ~(size_t)255;
  std::map<int, int> zslab;  // slot of a Z value -> slab in b2pk
  int inv_tag = 0;
  for (const Step& st : S.steps) {
    if (st.kind == Step::INV) {
      for (size_t c0 = 0; c0 < st.inv.size(); c0 += X.inv_chunk) {
        const size_t c1 = std::min(st.inv.size(), c0 + (size_t)X.inv_chunk);
        const size_t o = take((c1 - c0) * sizeof(InvDesc));
        InvDesc* hd = (InvDesc*)(hbase + o);
        int in_dt = -1, out_dt = -1;
        for (size_t t = c0; t < c1; ++t) {
          InvDesc d{};
          int64_t ld;
          d.src = resolve(c, st.inv[t].src, X, &ld, &in_dt);
          d.lds = ld;
          d.dst = (void*)resolve(c, st.inv[t].dst, X, &ld, &out_dt);
          d.ldd = ld;
          d.work = (char*)c->inv_work.p + (t - c0) * wstride;
          d.wrow = (char*)c->inv_wrow.p + (t - c0) * rstride;
          d.perm = (int*)((char*)c->inv_perm.p + (t - c0) * pstride);
          d.amax = (unsigned long long*)((char*)c->inv_amax.p + (t - c0) * 256);
          d.b = b;
          d.tag = inv_tag++;
          hd[t - c0] = d;
        }
        L.push_back({0, o, (int)(c1 - c0), in_dt, out_dt, 0, 0, nullptr, nullptr});
      }
      continue;
    }
    if (st.gemm.empty()) continue;
    const bool second = st.gemm[0].Cin.kind != Ref::NONE;  // X = K - L Z
    // distinct A operands
    std::map<std::pair<int, int>, int> aslab;
    std::vector<const GemmOp*> afirst;
    for (const GemmOp& g : st.gemm) {
      auto key = std::make_pair(g.A.kind == Ref::SLOT ? g.A.slot : -1 - g.A.r, g.A.c);
      if (aslab.emplace(key, (int)afirst.size()).second) afirst.push_back(&g);
    }
    {
      const size_t o = take(afirst.size() * sizeof(tc::PackDesc));
      tc::PackDesc* pd = (tc::PackDesc*)(hbase + o);
      for (size_t t = 0; t < afirst.size(); ++t) {
        int64_t ld;
        int dt;
        const void* p = resolve(c, afirst[t]->A, X, &ld, &dt);
        pd[t] = tc::PackDesc{p, ld, b, b, dt == F64 ? 1 : 0, 0, (int)t};
      }
      L.push_back({1, o, (int)afirst.size(), 0, 0, 0, 0, (__nv_bfloat16*)c->apk.p, nullptr});
    }
    if (!second) {
      // B = R^T slices, one slab per product
      const size_t o = take(st.gemm.size() * sizeof(tc::PackDesc));
      tc::PackDesc* pd = (tc::PackDesc*)(hbase + o);
      for (size_t t = 0; t < st.gemm.size(); ++t) {
        int64_t ld;
        int dt;
        const void* p = resolve(c, st.gemm[t].B, X, &ld, &dt);
        pd[t] = tc::PackDesc{p, ld, b, b, dt == F64 ? 1 : 0, 1, (int)t};
      }
      L.push_back({2, o, (int)st.gemm.size(), 0, 0, 0, 0, (__nv_bfloat16*)c->bpk.p, nullptr});
    }
    const size_t o = take(st.gemm.size() * sizeof(tc::TcProblem));
    tc::TcProblem* pr = (tc::TcProblem*)(hbase + o);
    for (size_t t = 0; t < st.gemm.size(); ++t) {
      const GemmOp& g = st.gemm[t];
      tc::TcProblem q{};
      q.a_slab = aslab[std::make_pair(g.A.kind == Ref::SLOT ? g.A.slot : -1 - g.A.r, g.A.c)];
      if (!second) {
        q.b_slab = (int)t;
        q.out_slab = (int)t;
        zslab[g.C.slot] = (int)t;
      } else {
        auto it = zslab.find(g.B.slot);
        if (g.B.kind != Ref::SLOT || it == zslab.end()) return MBINV_ENOTSUP;
        q.b_slab = it->second;
        int64_t ld;
        int dt;
        q.cin = resolve(c, g.Cin, X, &ld, &dt);
        q.ldcin = ld;
        q.cin_f64 = dt == F64 ? 1 : 0;
        q.out = (void*)resolve(c, g.C, X, &ld, &dt);
        q.ldo = ld;
        if (dt != F32) return MBINV_ENOTSUP;
      }
      pr[t] = q;
    }
    Launch l{3, o, (int)st.gemm.size(), 0, 0, (int)afirst.size(), second ? 0 : 1, (__nv_bfloat16*)c->apk.p,
             (__nv_bfloat16*)(second ? c->b2pk.p : c->bpk.p)};
    L.push_back(l);
  }
  if (off + 2 * sizeof(DevStatus) > need) return MBINV_ENOTSUP;
  CU(cudaMemcpyAsync(dbase, hbase, off, cudaMemcpyHostToDevice, c->stream));
  DevStatus* hst = (DevStatus*)(hbase + need - sizeof(DevStatus) * 2);
  hst[0] = DevStatus{0, INT_MAX};
  CU(cudaMemcpyAsync(c->status.p, &hst[0], sizeof(DevStatus), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemsetAsync(c->tcerr.p, 0, sizeof(int), c->stream));
  const bool prof = c->opt.profile != 0;
  if (prof) CU(ensure_events(c, 2 * L.size()));
  tc::TcParams P{};
  P.m = P.n = b;
  P.kpad = kpad;
  P.tiles_m = P.tiles_n = rpad / T;
  P.S = NS;
  tc::pair_table(NS, &P.npairs, P.pa, P.pb);
  P.orows = rpad;
  P.okpad = kpad;
  P.opk = (__nv_bfloat16*)c->b2pk.p;
  P.err = (int*)c->tcerr.p;
  for (size_t q = 0; q < L.size(); ++q) {
    const Launch& l = L[q];
    if (prof) CU(cudaEventRecord(c->events[2 * q], c->stream));
    switch (l.kind) {
      case 0:
        CU(run_inverse_batch(l.in_dt, l.out_dt, F64, (const InvDesc*)(dbase + l.off), l.count, b,
                             (DevStatus*)c->status.p, c->stream, &X.launches));
        break;
      case 1:
      case 2:
        CU(tc::launch_pack((const tc::PackDesc*)(dbase + l.off), l.count, NS, rpad, kpad, l.adst, c->stream));
        ++X.launches;
        break;
      case 3: {
        P.mode = l.mode;
        P.alpha = l.mode == 0 ? -1.f : 1.f;
        P.beta = 1.f;
        CU(tc::launch_gemm(l.adst, l.nA, rpad, l.bsrc, l.count, rpad, P, (const tc::TcProblem*)(dbase + l.off),
                           l.count, c->stream));
        ++X.launches;
        ++X.gemm_launches;
        break;
      }
    }
    if (prof) CU(cudaEventRecord(c->events[2 * q + 1], c->stream));
  }
  int* herr = (int*)&hst[1].tag;  // reuse the pinned words
  CU(cudaMemcpyAsync(&hst[1], c->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  const DevStatus st = hst[1];
  CU(cudaMemcpyAsync(herr, c->tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (*herr) return MBINV_ETIMEOUT;
  if (prof) {
    for (size_t q = 0; q < L.size(); ++q) {
      float ms = 0;
      CU(cudaEventElapsedTime(&ms, c->events[2 * q], c->events[2 * q + 1]));
      if (L[q].kind == 0) X.inv_dev_s += ms * 1e-3;
      else if (L[q].kind == 3) X.gemm_dev_s += ms * 1e-3;
      else X.pack_dev_s += ms * 1e-3;
    }
  }
  if (st.singular) return MBINV_ESINGULAR;
  return MBINV_OK;
}

mbinv_status prepare_border(mbinv_ctx* c, int64_t i, int64_t j) {
  if (c->l == 0) return MBINV_OK;
  int mode = 0;
  if (i != j && j == c->k - 1) mode = 1;
  else if (i != j && i == c->k - 1) mode = 2;
  if (mode == c->border_mode) return MBINV_OK;
  const int64_t nel = c->n * c->l;
  const int threads = 256;
  const int blocks = (int)((nel + threads - 1) / threads);
  if (c->mdt == F64)
    border_kernel<double><<<blocks, threads, 0, c->stream>>>((double*)c->dM, c->ldm, c->n, c->l, c->opt.pad_seed, mode);
  else
    border_kernel<float><<<blocks, threads, 0, c->stream>>>((float*)c->dM, c->ldm, c->n, c->l, c->opt.pad_seed, mode);
  CU(cudaGetLastError());
  c->border_mode = mode;
  return MBINV_OK;
}

void fill_report(mbinv_report* r, const mbinv_ctx* c, const Schedule& S, const Exec& X, double secs, size_t peak) {
  if (!r) return;
  const int launches = X.launches;
  r->gemm_device_seconds += X.gemm_dev_s;
  r->inv_device_seconds += X.inv_dev_s;
  r->gemm_launches += (size_t)X.gemm_launches;
  const double b3 = (double)c->b * (double)c->b * (double)c->b;
  r->gemm_flops += S.gemm_flops_units * b3;
  r->inv_flops += S.inv_units * b3;
  r->seconds += secs;
  r->peak_device_bytes = std::max(r->peak_device_bytes, peak);
  r->frames += S.frames;
  r->inversions += S.inversions;
  r->launches += (size_t)launches;
}

// One block into a device buffer dst (b x b, leading dimension ldd, dtype of M).
mbinv_status block_to_device(mbinv_ctx* c, int64_t i, int64_t j, void* dst, int64_t ldd, mbinv_report* rep) {
  auto t0 = std::chrono::steady_clock::now();
  mbinv_status s = prepare_border(c, i, j);
  if (s != MBINV_OK) return s;
  if (c->k == 1) {
    // the recursion degenerates to one inversion of M
    Schedule S;
    Step st;
    st.kind = Step::INV;
    InvOp io;
    io.src.kind = Ref::MBLK;
    io.dst.kind = Ref::OUT;
    st.inv.push_back(io);
    S.steps.push_back(st);
    S.inv_units = 2;
    S.inversions = 1;
    S.max_inv_batch = 1;
    if (c->opt.device_cap_bytes && c->own_M.bytes + schedule_bytes(c, S, 1) > c->opt.device_cap_bytes)
      return MBINV_ENOMEM_CAP;
    s = ensure_workspace(c, S, 1);
    if (s != MBINV_OK) return s;
    Exec X{c, &S, dst, ldd, c->dtype, 1};
    s = run_schedule(X);
    auto t1 = std::chrono::steady_clock::now();
    fill_report(rep, c, S, X, std::chrono::duration<double>(t1 - t0).count(), c->own_bytes);
    return s;
  }
  auto key = std::make_pair((int)i, (int)j);
  auto it = c->plans.find(key);
  if (it == c->plans.end()) {
    Plan P = build_plan((int)c->k, (int)i, (int)j, c->l > 0);
    Schedule S;
    int ic;
    if (!fit_cap(c, P, &S, &ic)) return MBINV_ENOMEM_CAP;
    S.max_inv_batch = ic;  // reuse the field: the chosen inverse chunk
    if (c->plans.size() > 4096) c->plans.clear();
    it = c->plans.emplace(key, std::make_pair(std::move(P), std::move(S))).first;
  }
  const Schedule& S = it->second.second;
  const int ic = std::max(1, S.max_inv_batch);
  s = ensure_workspace(c, S, ic);
  if (s != MBINV_OK) return s;
  Exec X{c, &S, dst, ldd, c->dtype, ic};
  s = c->opt.precision == MBINV_MIXED_BF16 ? run_schedule_mixed(X) : run_schedule(X);
  auto t1 = std::chrono::steady_clock::now();
  fill_report(rep, c, S, X, std::chrono::duration<double>(t1 - t0).count(), c->own_bytes);
  return s;
}

int64_t block_extent(const mbinv_ctx* c, int64_t t) {
  return (t == c->k - 1) ? c->n - (c->k - 1) * c->b : c->b;
}

// Copies rows x cols of a device buffer into out (host or device).
mbinv_status copy_out(mbinv_ctx* c, const void* src, int64_t lds, void* out, int64_t ldo, int64_t rows, int64_t cols,
                      bool out_dev) {
  const size_t es = dtype_size(c->dtype);
  CU(cudaMemcpy2DAsync(out, (size_t)ldo * es, src, (size_t)lds * es, (size_t)cols * es, (size_t)rows,
                       out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return MBINV_OK;
}

}  // namespace

// ====================================================================== ABI

extern "C" mbinv_status mbinv_refined_block_internal(mbinv_ctx* c, int64_t i, int64_t j, void* out, int64_t ldo,
                                                     mbinv_report* rep);

extern "C" {

void mbinv_default_options(mbinv_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->struct_size = sizeof *opt;
  opt->precision = MBINV_FP64;
  opt->device_cap_bytes = 0;
  opt->refine_steps = 0;
  opt->bf16_slices = 3;
  opt->cuda_stream = nullptr;
  opt->pad_seed = 0;
}

const char* mbinv_status_string(mbinv_status s) {
  switch (s) {
    case MBINV_OK: return "ok";
    case MBINV_EINVAL: return "invalid argument";
    case MBINV_ENOMEM_CAP: return "plan does not fit the device memory cap";
    case MBINV_ESINGULAR: return "a pivot block the recursion must invert is singular";
    case MBINV_ENOTCONV: return "refinement did not converge";
    case MBINV_ETIMEOUT: return "a device wait timed out";
    case MBINV_ECUDA: return "CUDA error";
    case MBINV_ENOTSUP: return "unsupported combination";
  }
  return "unknown status";
}

const char* mbinv_version(void) { return "mbinv 0.1 (sm_103a)"; }

const char* mbinv_last_cuda_error(void) { return cudaGetErrorString(last_cuda_error()); }

mbinv_status mbinv_create(mbinv_ctx** out, int64_t n, int64_t k, int dtype, const void* M, int64_t ld,
                          const mbinv_options* opt) {
  if (!out || !M || n <= 0 || k <= 0 || k > 63 || k > n || ld < n || (dtype != F64 && dtype != F32))
    return MBINV_EINVAL;
  *out = nullptr;
  mbinv_options o;
  mbinv_default_options(&o);
  if (opt) {
    if (opt->struct_size != sizeof(mbinv_options)) return MBINV_EINVAL;
    o = *opt;
  }
  if (o.precision < MBINV_FP64 || o.precision > MBINV_MIXED_BF16) return MBINV_EINVAL;
  if (o.precision == MBINV_MIXED_BF16 && (o.bf16_slices < 1 || o.bf16_slices > 3)) return MBINV_EINVAL;
  if (o.refine_steps < 0 || o.refine_steps > 1) return MBINV_EINVAL;
  std::unique_ptr<mbinv_ctx> c(new (std::nothrow) mbinv_ctx);
  if (!c) return MBINV_EINVAL;
  c->n = n;
  c->k = k;
  c->b = (n + k - 1) / k;
  c->npad = c->b * k;
  c->l = c->npad - n;
  c->dtype = dtype;
  c->opt = o;
  c->stream = (cudaStream_t)o.cuda_stream;
  // the plain paths read M in their own precision; the mixed path reads the
  // caller's M as given (its residual is taken against it)
  c->mdt = (o.precision == MBINV_FP64) ? F64 : (o.precision == MBINV_FP32 ? F32 : dtype);
  const size_t es = dtype_size(dtype), mes = dtype_size(c->mdt);
  const bool dev = is_device_ptr(M);
  if (c->l == 0 && dev && c->mdt == dtype) {
    c->dM = M;
    c->ldm = ld;
  } else {
    const size_t mbytes = (size_t)c->npad * c->npad * mes;
    if (o.device_cap_bytes && mbytes > o.device_cap_bytes) return MBINV_ENOMEM_CAP;
    CU(c->own_M.ensure(mbytes));
    c->dM = c->own_M.p;
    c->ldm = c->npad;
    if (c->mdt == dtype) {
      CU(cudaMemcpy2DAsync(c->own_M.p, (size_t)c->npad * mes, M, (size_t)ld * es, (size_t)n * es, (size_t)n,
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    } else {
      // stage the caller's matrix on the device, then convert it
      DevBuf stage;
      CU(stage.ensure((size_t)n * n * es));
      CU(cudaMemcpy2DAsync(stage.p, (size_t)n * es, M, (size_t)ld * es, (size_t)n * es, (size_t)n,
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
      const int64_t nel = n * n;
      const int blocks = (int)((nel + 255) / 256);
      if (dtype == F64)
        convert_kernel<double, float><<<blocks, 256, 0, c->stream>>>((const double*)stage.p, n, (float*)c->own_M.p,
                                                                      c->npad, n, n);
      else
        convert_kernel<float, double><<<blocks, 256, 0, c->stream>>>((const float*)stage.p, n, (double*)c->own_M.p,
                                                                      c->npad, n, n);
      CU(cudaGetLastError());
      CU(cudaStreamSynchronize(c->stream));
      stage.release();
    }
    if (c->l) {
      // identity in the padded corner; the border strips are written per request
      std::vector<char> eye((size_t)c->l * c->npad * mes, 0);
      for (int64_t q = 0; q < c->l; ++q) {
        if (c->mdt == F64) ((double*)eye.data())[q * c->npad + n + q] = 1.0;
        else ((float*)eye.data())[q * c->npad + n + q] = 1.0f;
      }
      CU(cudaMemcpyAsync((char*)c->own_M.p + (size_t)n * c->npad * mes, eye.data(), eye.size(),
                         cudaMemcpyHostToDevice, c->stream));
      CU(cudaStreamSynchronize(c->stream));
      mbinv_status s = prepare_border(c.get(), 0, 0);
      if (s != MBINV_OK) return s;
    }
    CU(cudaStreamSynchronize(c->stream));
  }
  *out = c.release();
  return MBINV_OK;
}

void mbinv_destroy(mbinv_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  for (DevBuf* d : {&c->own_M, &c->slots, &c->inv_work, &c->inv_wrow, &c->inv_perm, &c->inv_amax, &c->desc,
                    &c->status, &c->outtmp, &c->rowbuf, &c->colbuf, &c->resid, &c->apk, &c->bpk, &c->b2pk,
                    &c->tcerr})
    d->release();
  c->hdesc.release();
  c->hstage.release();
  delete c;
}

mbinv_status mbinv_block(mbinv_ctx* c, int64_t i, int64_t j, void* out, int64_t ldo, mbinv_report* rep) {
  if (!c || !out || i < 0 || j < 0 || i >= c->k || j >= c->k) return MBINV_EINVAL;
  const int64_t bi = block_extent(c, i), bj = block_extent(c, j);
  if (ldo < bj) return MBINV_EINVAL;
  if (rep) {
    std::memset(rep, 0, sizeof *rep);
    rep->failed_pivot = -1;
  }
  if (c->opt.precision == MBINV_MIXED_BF16 && c->opt.refine_steps > 0 && !c->in_sweep) {
    auto t0 = std::chrono::steady_clock::now();
    c->in_sweep = true;
    mbinv_status r = mbinv_refined_block_internal(c, i, j, out, ldo, rep);
    c->in_sweep = false;
    if (rep) rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return r;
  }
  const bool out_dev = is_device_ptr(out);
  mbinv_status s;
  if (out_dev && bi == c->b && bj == c->b) {
    s = block_to_device(c, i, j, out, ldo, rep);
  } else {
    CU(c->outtmp.ensure((size_t)c->b * c->b * 8 + 256));
    s = block_to_device(c, i, j, c->outtmp.p, c->b, rep);
    if (s == MBINV_OK) s = copy_out(c, c->outtmp.p, c->b, out, ldo, bi, bj, out_dev);
  }
  return s;
}

mbinv_status mbinv_all_blocks(mbinv_ctx* c, void* out, int64_t ldo, const uint8_t* done, mbinv_block_done_cb cb,
                              void* user, mbinv_report* rep) {
  if (!c || !out || ldo < c->n) return MBINV_EINVAL;
  mbinv_report acc;
  std::memset(&acc, 0, sizeof acc);
  acc.failed_pivot = -1;
  const size_t es = dtype_size(c->dtype);
  for (int64_t i = 0; i < c->k; ++i)
    for (int64_t j = 0; j < c->k; ++j) {
      if (done && done[i * c->k + j]) continue;
      mbinv_report r;
      void* dst = (char*)out + ((size_t)i * c->b * ldo + (size_t)j * c->b) * es;
      mbinv_status s = mbinv_block(c, i, j, dst, ldo, &r);
      if (s != MBINV_OK) {
        if (rep) *rep = acc;
        return s;
      }
      acc.gemm_flops += r.gemm_flops;
      acc.inv_flops += r.inv_flops;
      acc.seconds += r.seconds;
      acc.frames += r.frames;
      acc.inversions += r.inversions;
      acc.launches += r.launches;
      acc.gemm_launches += r.gemm_launches;
      acc.gemm_device_seconds += r.gemm_device_seconds;
      acc.inv_device_seconds += r.inv_device_seconds;
      acc.peak_device_bytes = std::max(acc.peak_device_bytes, r.peak_device_bytes);
      if (cb) cb(i, j, user);
    }
  if (rep) *rep = acc;
  return MBINV_OK;
}

static mbinv_status row_or_col(mbinv_ctx* c, int64_t t, bool row, void* out, int64_t ldo, mbinv_report* rep) {
  if (!c || !out || t < 0 || t >= c->k) return MBINV_EINVAL;
  if (ldo < (row ? c->n : block_extent(c, t))) return MBINV_EINVAL;
  mbinv_report acc;
  std::memset(&acc, 0, sizeof acc);
  acc.failed_pivot = -1;
  const size_t es = dtype_size(c->dtype);
  for (int64_t q = 0; q < c->k; ++q) {
    const int64_t i = row ? t : q, j = row ? q : t;
    void* dst = row ? (char*)out + (size_t)q * c->b * es : (char*)out + (size_t)q * c->b * ldo * es;
    mbinv_report r;
    mbinv_status s = mbinv_block(c, i, j, dst, ldo, &r);
    if (s != MBINV_OK) return s;
    acc.gemm_flops += r.gemm_flops;
    acc.inv_flops += r.inv_flops;
    acc.seconds += r.seconds;
    acc.frames += r.frames;
    acc.inversions += r.inversions;
    acc.launches += r.launches;
    acc.gemm_launches += r.gemm_launches;
    acc.gemm_device_seconds += r.gemm_device_seconds;
    acc.inv_device_seconds += r.inv_device_seconds;
    acc.peak_device_bytes = std::max(acc.peak_device_bytes, r.peak_device_bytes);
  }
  if (rep) *rep = acc;
  return MBINV_OK;
}

mbinv_status mbinv_block_row(mbinv_ctx* c, int64_t i, void* out, int64_t ldo, mbinv_report* rep) {
  return row_or_col(c, i, true, out, ldo, rep);
}

mbinv_status mbinv_block_col(mbinv_ctx* c, int64_t j, void* out, int64_t ldo, mbinv_report* rep) {
  return row_or_col(c, j, false, out, ldo, rep);
}

}  // extern "C"

namespace {

mbinv_status gemm1(mbinv_ctx* c, int combo, const void* A, int64_t lda, int ta, const void* B, int64_t ldb, int tb,
                   const void* Cin, int64_t ldcin, void* C, int64_t ldc, int m, int n, int k, double alpha,
                   double beta) {
  GemmDesc d{};
  d.A = A;
  d.lda = lda;
  d.ta = ta;
  d.B = B;
  d.ldb = ldb;
  d.tb = tb;
  d.Cin = Cin;
  d.ldcin = ldcin;
  d.C = C;
  d.ldc = ldc;
  d.m = m;
  d.n = n;
  d.k = k;
  d.alpha = alpha;
  d.beta = beta;
  int bm, bn;
  gemm_tile_shape(combo, &bm, &bn);
  d.tiles_n = (n + bn - 1) / bn;
  d.tile_start = 0;
  const int tiles = ((m + bm - 1) / bm) * d.tiles_n;
  CU(c->desc.ensure(4096));
  CU(c->hdesc.ensure(4096));
  std::memcpy(c->hdesc.p, &d, sizeof d);
  CU(cudaMemcpyAsync(c->desc.p, c->hdesc.p, sizeof d, cudaMemcpyHostToDevice, c->stream));
  CU(launch_gemm_grouped(combo, (const GemmDesc*)c->desc.p, 1, tiles, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return MBINV_OK;
}

}  // namespace

extern "C" {

mbinv_status mbinv_backward(mbinv_ctx* c, int64_t i, int64_t j, const void* G, int64_t ldg, void* dM, int64_t ldd,
                            mbinv_report* rep) {
  if (!c || !G || !dM || i < 0 || j < 0 || i >= c->k || j >= c->k || ldd < c->n) return MBINV_EINVAL;
  const int64_t bi = block_extent(c, i), bj = block_extent(c, j), n = c->n;
  if (ldg < bj) return MBINV_EINVAL;
  const size_t es = dtype_size(c->dtype);
  const int combo = c->dtype == F64 ? G_F64 : G_F32;
  // X_i (bi x n) and Y_j (n x bj) of M^-1, block by block
  CU(c->rowbuf.ensure((size_t)bi * n * es + 256));
  CU(c->colbuf.ensure((size_t)n * bj * es + 256));
  mbinv_report r1, r2;
  mbinv_status s = mbinv_block_row(c, i, c->rowbuf.p, n, &r1);
  if (s != MBINV_OK) return s;
  s = mbinv_block_col(c, j, c->colbuf.p, bj, &r2);
  if (s != MBINV_OK) return s;
  // G and dM on the device
  DevBuf gdev, ddev, wbuf;
  const void* Gd = G;
  if (!is_device_ptr(G)) {
    CU(gdev.ensure((size_t)bi * bj * es));
    CU(cudaMemcpy2DAsync(gdev.p, (size_t)bj * es, G, (size_t)ldg * es, (size_t)bj * es, (size_t)bi,
                         cudaMemcpyHostToDevice, c->stream));
    Gd = gdev.p;
    ldg = bj;
  }
  void* Dd = dM;
  int64_t lddd = ldd;
  const bool dm_host = !is_device_ptr(dM);
  if (dm_host) {
    CU(ddev.ensure((size_t)n * n * es));
    CU(cudaMemcpy2DAsync(ddev.p, (size_t)n * es, dM, (size_t)ldd * es, (size_t)n * es, (size_t)n,
                         cudaMemcpyHostToDevice, c->stream));
    Dd = ddev.p;
    lddd = n;
  }
  // W = G Y_j^T (bi x n), then dM += -X_i^T W
  CU(wbuf.ensure((size_t)bi * n * es));
  s = gemm1(c, combo, Gd, ldg, 0, c->colbuf.p, bj, 1, nullptr, 0, wbuf.p, n, (int)bi, (int)n, (int)bj, 1.0, 0.0);
  if (s != MBINV_OK) return s;
  s = gemm1(c, combo, c->rowbuf.p, n, 1, wbuf.p, n, 0, Dd, lddd, Dd, lddd, (int)n, (int)n, (int)bi, -1.0, 1.0);
  if (s != MBINV_OK) return s;
  if (dm_host) {
    CU(cudaMemcpy2DAsync(dM, (size_t)ldd * es, ddev.p, (size_t)n * es, (size_t)n * es, (size_t)n,
                         cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  if (rep) {
    std::memset(rep, 0, sizeof *rep);
    rep->failed_pivot = -1;
    rep->gemm_flops = r1.gemm_flops + r2.gemm_flops + 2.0 * bi * bj * n + 2.0 * n * n * bi;
    rep->inv_flops = r1.inv_flops + r2.inv_flops;
    rep->seconds = r1.seconds + r2.seconds;
    rep->frames = r1.frames + r2.frames;
    rep->inversions = r1.inversions + r2.inversions;
    rep->launches = r1.launches + r2.launches + 2;
    rep->peak_device_bytes = std::max(r1.peak_device_bytes, r2.peak_device_bytes) + c->rowbuf.bytes + c->colbuf.bytes;
  }
  return MBINV_OK;
}

mbinv_status mbinv_batched_blocks(int64_t count, mbinv_problem* probs, int dtype, const mbinv_options* opt,
                                  mbinv_report* rep) {
  if (count < 0 || (count > 0 && !probs)) return MBINV_EINVAL;
  mbinv_status first = MBINV_OK;
  if (rep) {
    std::memset(rep, 0, sizeof *rep);
    rep->failed_pivot = -1;
  }
  for (int64_t t = 0; t < count; ++t) {
    mbinv_problem& p = probs[t];
    mbinv_ctx* c = nullptr;
    mbinv_status s = mbinv_create(&c, p.n, p.k, dtype, p.M, p.ld, opt);
    if (s == MBINV_OK) {
      mbinv_report r;
      s = mbinv_block(c, p.i, p.j, p.out, p.ldo, &r);
      if (rep && s == MBINV_OK) {
        rep->gemm_flops += r.gemm_flops;
        rep->inv_flops += r.inv_flops;
        rep->seconds += r.seconds;
        rep->frames += r.frames;
        rep->inversions += r.inversions;
        rep->launches += r.launches;
        rep->peak_device_bytes = std::max(rep->peak_device_bytes, r.peak_device_bytes);
      }
      mbinv_destroy(c);
    }
    p.status = s;
    if (s != MBINV_OK && first == MBINV_OK) first = s;
  }
  return first;
}

}  // extern "C"

namespace {

// Mixed path with one two-sided refinement step:
//   X_i = block row i, Y_j = block column j of M^-1 from the mixed sweep,
//   R   = E_i^T - X_i M                      (FP64 accumulation)
//   N_ij <- X_i E_j + R Y_j                  (FP64)
// With dX, dY the errors of X_i, Y_j the result differs from N_ij by
// -dX M dY: the error is squared when it is small.
mbinv_status refined_block(mbinv_ctx* c, int64_t i, int64_t j, void* out, int64_t ldo, mbinv_report* rep) {
  const int64_t n = c->n, b = c->b;
  const int64_t bi = block_extent(c, i), bj = block_extent(c, j);
  // sweeps in FP32, straight into device buffers
  CU(c->rowbuf.ensure((size_t)b * n * 4 + 256));
  CU(c->colbuf.ensure((size_t)n * b * 4 + 256));
  CU(c->resid.ensure((size_t)b * n * 8 + (size_t)b * b * 8 + 512));
  const int saved_dtype = c->dtype;
  c->dtype = F32;  // the sweeps write FP32 blocks
  mbinv_report r1{}, r2{};
  mbinv_status s = mbinv_block_row(c, i, c->rowbuf.p, n, &r1);
  if (s == MBINV_OK) s = mbinv_block_col(c, j, c->colbuf.p, b, &r2);
  c->dtype = saved_dtype;
  if (s != MBINV_OK) return s;
  double* R = (double*)c->resid.p;                      // bi x n
  double* Nij = R + (size_t)b * n;                      // bi x bj
  double* acc = Nij + (size_t)b * b;
  const int cm = c->mdt == F64 ? G_F32F64_F64 : G_F32IN_F64;
  // R = -X_i M, then + E_i^T
  s = gemm1(c, cm, c->rowbuf.p, n, 0, c->dM, c->ldm, 0, nullptr, 0, R, n, (int)bi, (int)n, (int)n, -1.0, 0.0);
  if (s != MBINV_OK) return s;
  add_eye_kernel<<<(unsigned)((bi + 255) / 256), 256, 0, c->stream>>>(R, n, i * b, bi);
  CU(cudaGetLastError());
  CU(cudaMemsetAsync(acc, 0, sizeof(double), c->stream));
  sumsq_kernel<<<64, 256, 0, c->stream>>>(R, n, bi, n, acc);
  CU(cudaGetLastError());
  // N_ij = X_i E_j (FP32 -> FP64) + R Y_j
  convert_kernel<float, double><<<(unsigned)((bi * bj + 255) / 256), 256, 0, c->stream>>>(
      (const float*)c->rowbuf.p + j * b, n, Nij, bj, bi, bj);
  CU(cudaGetLastError());
  s = gemm1(c, G_F64F32_F64, R, n, 0, c->colbuf.p, b, 0, Nij, bj, Nij, bj, (int)bi, (int)bj, (int)n, 1.0, 1.0);
  if (s != MBINV_OK) return s;
  double hacc = 0;
  CU(cudaMemcpyAsync(&hacc, acc, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  // write out in the caller's dtype and memory
  const bool out_dev = is_device_ptr(out);
  const size_t es = dtype_size(c->dtype);
  if (c->dtype == F64) {
    CU(cudaMemcpy2DAsync(out, (size_t)ldo * es, Nij, (size_t)bj * 8, (size_t)bj * 8, (size_t)bi,
                         out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  } else {
    CU(c->outtmp.ensure((size_t)b * b * 8 + 256));
    convert_kernel<double, float><<<(unsigned)((bi * bj + 255) / 256), 256, 0, c->stream>>>(
        Nij, bj, (float*)c->outtmp.p, bj, bi, bj);
    CU(cudaGetLastError());
    CU(cudaMemcpy2DAsync(out, (size_t)ldo * es, c->outtmp.p, (size_t)bj * 4, (size_t)bj * 4, (size_t)bi,
                         out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  }
  CU(cudaStreamSynchronize(c->stream));
  if (rep) {
    rep->gemm_flops = r1.gemm_flops + r2.gemm_flops + 2.0 * bi * n * n + 2.0 * bi * bj * n;
    rep->inv_flops = r1.inv_flops + r2.inv_flops;
    rep->frames = r1.frames + r2.frames;
    rep->inversions = r1.inversions + r2.inversions;
    rep->launches = r1.launches + r2.launches + 5;
    rep->gemm_launches = r1.gemm_launches + r2.gemm_launches;
    rep->gemm_device_seconds = r1.gemm_device_seconds + r2.gemm_device_seconds;
    rep->inv_device_seconds = r1.inv_device_seconds + r2.inv_device_seconds;
    rep->peak_device_bytes = std::max(r1.peak_device_bytes, r2.peak_device_bytes) + c->rowbuf.bytes +
                             c->colbuf.bytes + c->resid.bytes;
    rep->rel_residual = std::sqrt(hacc / (double)bi);
  }
  if (!(std::sqrt(hacc / (double)bi) < 1.0)) return MBINV_ENOTCONV;
  return MBINV_OK;
}

}  // namespace

extern "C" mbinv_status mbinv_refined_block_internal(mbinv_ctx* c, int64_t i, int64_t j, void* out, int64_t ldo,
                                                     mbinv_report* rep) {
  return refined_block(c, i, j, out, ldo, rep);
}
