// C ABI of libmbinv.
//
// A request for block (i, j) is planned on the host (the forward procedure of
// Sec. 3.1 has no arithmetic) and run level by level on one CUDA stream
// (Sec. 3.2).  Independent requests - the k^2 runs of Sec. 5, a block row, a
// block column, many matrices - are run together: step t of every request's
// schedule goes out in the same grouped launches (exec.cu).  Values live in
// fixed-size b x b slots; each request has its own slot region, sized by the
// planner's liveness simulation, and the number of requests run together is
// bounded by the caller's device memory cap.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "../../include/mbinv.h"
#include "exec.h"
#include "mbinv_internal.h"
#include "ozaki.h"

using namespace mbinv;

namespace {

cudaError_t& last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

// A CUDA error becomes MBINV_ECUDA, except an allocation the cap refused,
// which becomes MBINV_ENOMEM_CAP.
#define CU(x)                                                \
  do {                                                       \
    cudaError_t e_ = (x);                                    \
    if (e_ != cudaSuccess) {                                 \
      if (e_ == cudaErrorMemoryAllocation && cap_refused()) { \
        cap_refused() = false;                               \
        return MBINV_ENOMEM_CAP;                             \
      }                                                      \
      last_cuda_error() = e_;                                \
      return MBINV_ECUDA;                                    \
    }                                                        \
  } while (0)

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

// Border strips of the bordered matrix: rows [0, n) x columns [n, n + l) hold
// B'[r][q] (mode 1, requests (i, k-1)), rows [n, n+l) x columns [0, n) hold
// C'[q][r] = B'[r][q] (mode 2, requests (k-1, j)); zero otherwise.
// B'[r][q] = uniform[-1, 1) draw r*l + q of stream 6.
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
  g[r * ldg + n + q] = (mode == 1) ? (T)v : (T)0;
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

}  // namespace

struct mbinv_ctx {
  int64_t n = 0, k = 0, b = 0, npad = 0, l = 0;
  int dtype = F64;  // the caller's element type (M, G, dM)
  int odt = F64;    // element type of the returned blocks
  int mdt = F64;    // element type of the device matrix the sweep reads
  mbinv_options opt{};
  cudaStream_t stream = nullptr;
  const void* dM = nullptr;  // borrowed caller pointer, or own_M
  int64_t ldm = 0;
  const void* hM = nullptr;  // host-resident M (bounded schedule): borrowed, caller's dtype
  int64_t hld = 0;
  mbinv_block_fn gen = nullptr;  // produced M (bounded schedule): never stored
  void* gen_user = nullptr;
  HostBuf spill;             // pinned host slots of the values a bounded run spills
  const void* srcM = nullptr;  // the caller's M as given to create (borrowed), its ld and space
  int64_t srcld = 0;
  bool srcdev = false;
  DevBuf own_M;
  int border_mode = -1;
  DevBuf slots, outtmp, rowbuf, colbuf, resid, gbuf, wbuf, dmbuf, gemmdesc;
  Env env;
  MemTrack track;  // every device byte the context holds
  std::vector<DevBuf*> bufs() {
    std::vector<DevBuf*> v = {&own_M, &slots, &outtmp, &rowbuf, &colbuf, &resid, &gbuf, &wbuf, &dmbuf, &gemmdesc};
    for (DevBuf* d : env.bufs()) v.push_back(d);
    return v;
  }
  // the buffers of the sweep (value slots and the executor's workspace)
  std::vector<DevBuf*> sweep_bufs() {
    std::vector<DevBuf*> v = {&slots};
    for (DevBuf* d : env.bufs()) v.push_back(d);
    return v;
  }
  // plans by request group (the requests whose frames are merged)
  std::map<std::vector<std::pair<int, int>>, std::pair<Plan, Schedule>> plans;
  bool in_sweep = false;
  int depth = 0;  // nesting of entry-point calls on this context
};

namespace {

int64_t block_extent(const mbinv_ctx* c, int64_t t) { return (t == c->k - 1) ? c->n - (c->k - 1) * c->b : c->b; }

int border_of(const mbinv_ctx* c, int64_t i, int64_t j) {
  if (c->l == 0) return 0;
  if (i != j && j == c->k - 1) return 1;
  if (i != j && i == c->k - 1) return 2;
  return 0;
}

mbinv_status set_border(mbinv_ctx* c, int mode) {
  if (c->l == 0 || mode == c->border_mode) return MBINV_OK;
  const int64_t nel = c->n * c->l;
  const int blocks = (int)((nel + 255) / 256);
  if (c->mdt == F64)
    border_kernel<double><<<blocks, 256, 0, c->stream>>>((double*)c->dM, c->ldm, c->n, c->l, c->opt.pad_seed, mode);
  else
    border_kernel<float><<<blocks, 256, 0, c->stream>>>((float*)c->dM, c->ldm, c->n, c->l, c->opt.pad_seed, mode);
  CU(cudaGetLastError());
  c->border_mode = mode;
  return MBINV_OK;
}

// Inverse scratch is bounded even without a cap: at most this many matrices
// of order b go into one batched inverse launch sequence.
constexpr size_t kInvScratchBudget = 8ull << 30;
int max_inv_chunk(int b, int prec) {
  const size_t per = inv_scratch_bytes(b, prec, 1);
  return (int)std::max<size_t>(1, std::min<size_t>(1 << 20, kInvScratchBudget / per));
}

// Memory of running one (merged) schedule, beyond M.
size_t run_bytes(const mbinv_ctx* c, const Schedule& S, int inv_chunk) {
  const int prec = c->opt.precision;
  size_t bytes = (size_t)S.nslots * slot_bytes_for((int)c->b, prec) + 256;
  bytes += inv_scratch_bytes((int)c->b, prec, inv_chunk);
  // descriptors, operand slabs, staging: as the executor reckons them, plus
  // its status words
  bytes += arena_bytes(S, (int)c->b, prec, c->opt.bf16_slices, inv_chunk, c->dtype, env_slot_type(prec)) +
           (64u << 10);
  return bytes;
}

// Device bytes held outside the sweep's workspace (M, output staging,
// refinement buffers): what a sweep's plan must fit beside.
size_t base_bytes(mbinv_ctx* c) {
  // a context of a batched call counts into the call's tracker, with the
  // other problems: its plan fits beside its own matrix copy
  if (c->own_M.track != &c->track) return c->own_M.bytes;
  size_t sweep = 0;
  for (DevBuf* d : c->sweep_bufs()) sweep += d->bytes;
  return c->track.live - sweep;
}

// Under a cap, the sweep's workspace is freed between groups, so that its
// buffers never hold more than the plan of the group being run.
void release_sweep(mbinv_ctx* c) {
  if (!c->opt.device_cap_bytes) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (DevBuf* d : c->sweep_bufs()) d->release();
}

// The merged plan of a group of requests, with its Schur-temporary chunk and
// inverse chunk chosen to fit the cap beside what the context already holds.
mbinv_status get_plan(mbinv_ctx* c, const std::vector<std::pair<int, int>>& reqs, const Schedule** out) {
  auto it = c->plans.find(reqs);
  if (it != c->plans.end() &&
      (!c->opt.device_cap_bytes || base_bytes(c) + it->second.second.planned <= c->opt.device_cap_bytes)) {
    *out = &it->second.second;
    return MBINV_OK;
  }
  const size_t cap = c->opt.device_cap_bytes;
  const size_t base = base_bytes(c);
  if (c->k == 1) {
    // the recursion degenerates to one inversion of M per request
    Schedule S;
    Step st;
    st.kind = Step::INV;
    for (size_t r = 0; r < reqs.size(); ++r) {
      InvOp io;
      io.src.kind = Ref::MBLK;
      io.dst.kind = Ref::OUT;
      io.dst.slot = (int)r;
      st.inv.push_back(io);
    }
    S.steps.push_back(st);
    S.nouts = (int)reqs.size();
    S.inv_units = 2.0 * reqs.size();
    S.inversions = reqs.size();
    S.max_inv_batch = (int)reqs.size();
    S.frames = S.request_frames = 0;
    const int full = std::min<int>((int)reqs.size(), max_inv_chunk((int)c->b, c->opt.precision));
    bool ok = false;
    for (int ic : {full, 256, 64, 16, 4, 1}) {
      if (ic > full) continue;
      if (cap == 0 || base + run_bytes(c, S, ic) <= cap) {
        S.inv_chunk = ic;
        S.planned = run_bytes(c, S, ic);
        ok = true;
        break;
      }
    }
    if (!ok) return MBINV_ENOMEM_CAP;
    if (c->plans.size() > 256) c->plans.clear();
    it = c->plans.insert_or_assign(reqs, std::make_pair(Plan{}, std::move(S))).first;
    *out = &it->second.second;
    return MBINV_OK;
  }
  Plan P = build_plan((int)c->k, reqs, c->l > 0);
  Schedule best;
  bool ok = false;
  const bool want_bounded = c->hM || c->gen || c->opt.schedule == MBINV_SCHEDULE_BOUNDED;
  for (int z : {0, 256, 64, 16, 4, 1}) {
    if (want_bounded) break;
    Schedule T = build_schedule(P, z);
    const int full = std::min(std::max(1, T.max_inv_batch), max_inv_chunk((int)c->b, c->opt.precision));
    for (int ic : {full, 256, 64, 16, 4, 1}) {
      if (ic > full) continue;
      if (cap == 0 || base + run_bytes(c, T, ic) <= cap) {
        T.inv_chunk = ic;
        T.planned = run_bytes(c, T, ic);
        best = std::move(T);
        ok = true;
        break;
      }
    }
    if (ok) break;
  }
  if (!ok && c->opt.schedule == MBINV_SCHEDULE_LEVELS) return MBINV_ENOMEM_CAP;
  if (!ok) {
    // depth first in the slots the cap leaves, values spilled to the host
    if (c->opt.precision == MBINV_MIXED_BF16 || c->l > 0) return MBINV_ENOTSUP;
    const size_t sb = slot_bytes_for((int)c->b, c->opt.precision);
    Schedule T;
    const bool host_m = c->hM != nullptr || c->gen != nullptr;
    if (!build_bounded_schedule(P, (int)std::min<size_t>(1u << 20, 4 * P.f.size() + 64), host_m, &T))
      return MBINV_ENOTSUP;
    int slots = T.nslots;  // no spill at all
    for (int iter = 0; cap && iter < 8; ++iter) {
      const size_t need = base + run_bytes(c, T, 1);
      if (need <= cap && T.nslots <= slots) break;
      const size_t over = need > cap ? (need - cap + sb - 1) / sb + 1 : 0;
      slots = std::min(slots, T.nslots) - (int)over;
      if (slots < 6) return MBINV_ENOMEM_CAP;
      if (!build_bounded_schedule(P, slots, host_m, &T)) return MBINV_ENOMEM_CAP;
    }
    if (cap && base + run_bytes(c, T, 1) > cap) return MBINV_ENOMEM_CAP;
    T.inv_chunk = 1;
    T.planned = run_bytes(c, T, 1);
    best = std::move(T);
  }
  if (c->plans.size() > 256) c->plans.clear();
  it = c->plans.insert_or_assign(reqs, std::make_pair(std::move(P), std::move(best))).first;
  *out = &it->second.second;
  return MBINV_OK;
}

struct Req {
  int64_t i, j;
  void* dst;  // device, b x b (leading dimension ldd), caller dtype
  int64_t ldd;
};

// Device seconds and flop split of the last run of env (profile option).
void add_env_report(mbinv_report* r, const Env& env) {
  r->gemm_device_seconds += env.gemm_dev_s;
  r->inv_device_seconds += env.inv_dev_s;
  r->pack_device_seconds += env.pack_dev_s;
  r->pack_bytes += env.pack_bytes;
  r->inv_panel_device_seconds += env.inv_panel_dev_s;
  r->inv_panel_flops += env.inv_panel_flops;
  r->inv_update_flops += env.inv_update_flops;
  r->inv_panel_launches += env.inv_panel_launches;
}

void add_report(mbinv_report* r, const mbinv_ctx* c, const Schedule& S) {
  if (!r) return;
  const double b3 = (double)c->b * (double)c->b * (double)c->b;
  r->gemm_flops += S.gemm_flops_units * b3;
  r->inv_flops += S.inv_units * b3;
  r->frames += S.frames;
  r->request_frames += S.request_frames;
  r->inversions += S.inversions;
}

std::vector<std::pair<int, int>> group_key(const std::vector<Req>& reqs, size_t n) {
  std::vector<std::pair<int, int>> key;
  for (size_t q = 0; q < n && q < reqs.size(); ++q) key.emplace_back((int)reqs[q].i, (int)reqs[q].j);
  return key;
}

// Runs a group of requests with the same border as one merged schedule:
// frames that compute the same thing are evaluated once for all of them.
mbinv_status run_group(mbinv_ctx* c, const std::vector<Req>& reqs, mbinv_report* rep) {
  if (reqs.empty()) return MBINV_OK;
  mbinv_status s = set_border(c, border_of(c, reqs[0].i, reqs[0].j));
  if (s != MBINV_OK) return s;
  const Schedule* S;
  s = get_plan(c, group_key(reqs, reqs.size()), &S);
  if (s != MBINV_OK) return s;
  release_sweep(c);
  const size_t planned = c->track.live + S->planned;
  const int prec = c->opt.precision;
  const size_t sb = slot_bytes_for((int)c->b, prec);
  CU(c->slots.ensure((size_t)S->nslots * sb + 256));
  Job J;
  J.dM = c->dM;
  J.ldm = c->ldm;
  J.mdt = c->mdt;
  J.b = (int)c->b;
  J.slots = (char*)c->slots.p;
  J.slot_bytes = sb;
  J.slot_dt = env_slot_type(prec);
  J.out_dt = c->odt;
  J.S = S;
  if (S->bounded) {
    J.hM = c->hM;
    J.hldm = c->hld;
    J.hmdt = c->dtype;
    J.gen = c->gen;
    J.gen_user = c->gen_user;
    if (S->nspill > 0) {
      CU(c->spill.ensure((size_t)S->nspill * sb));
      J.spill = (char*)c->spill.p;
    }
  }
  for (const Req& r : reqs) {
    J.outs.push_back(r.dst);
    J.ldos.push_back(r.ldd);
  }
  c->env.stream = c->stream;
  c->env.precision = prec;
  c->env.slices = c->opt.bf16_slices;
  c->env.profile = c->opt.profile != 0;
  c->env.inv_chunk = std::max(1, S->inv_chunk);
  c->env.sing_tol = c->opt.sing_tol;
  c->env.pivot_cond = c->opt.pivot_cond != 0;
  c->env.use_graphs = c->opt.no_graphs == 0;
  const size_t replays0 = c->env.graph_replays;
  s = run_jobs(c->env, {J});
  if (s == MBINV_ECUDA) last_cuda_error() = c->env.last_error;
  if (rep) {
    add_report(rep, c, *S);
    rep->launches += (size_t)c->env.launches;
    rep->gemm_launches += (size_t)c->env.gemm_launches;
    add_env_report(rep, c->env);
    rep->planned_device_bytes = std::max(rep->planned_device_bytes, planned);
    rep->max_pivot_cond = std::max(rep->max_pivot_cond, c->env.max_cond);
    rep->graph_replays += c->env.graph_replays - replays0;
    rep->host_in_bytes += c->env.host_in_bytes;
    rep->host_out_bytes += c->env.host_out_bytes;
    rep->host_spill_bytes = std::max(rep->host_spill_bytes, (size_t)S->nspill * sb);
    if (s == MBINV_ESINGULAR && rep->failed_pivot < 0) rep->failed_pivot = c->env.failed_inverse;
  }
  return s;
}

// Largest number of the first requests of v (at most want) whose merged
// schedule fits the cap.
int fit_group(mbinv_ctx* c, const std::vector<Req>& v, int want) {
  for (int G = want; G > 1; G = G / 2) {
    const Schedule* S;
    if (get_plan(c, group_key(v, (size_t)G), &S) == MBINV_OK) return G;
  }
  return 1;
}

// The principal-Schur variant (Sec. 8's reformulation around M/A): each
// request its own schedule (the eliminated sets differ between blocks), the
// schedules of a group - all of one shape - executed together, step t of
// every request in the same grouped launches.
const Schedule* psc_plan(mbinv_ctx* c, int64_t i, int64_t j) {
  auto key = std::vector<std::pair<int, int>>{{(int)i, (int)j}, {-1, -1}};  // marks the variant
  auto it = c->plans.find(key);
  if (it == c->plans.end()) {
    Schedule S = build_psc_schedule((int)c->k, (int)i, (int)j);
    S.inv_chunk = 1;
    S.planned = run_bytes(c, S, 1);
    if (c->plans.size() > 256) c->plans.clear();
    it = c->plans.emplace(key, std::make_pair(Plan{}, std::move(S))).first;
  }
  return &it->second.second;
}

int fit_group_psc(mbinv_ctx* c, const std::vector<Req>& v, int want) {
  const size_t cap = c->opt.device_cap_bytes;
  if (!cap) return want;
  const size_t per = psc_plan(c, v[0].i, v[0].j)->planned;
  const size_t base = base_bytes(c);
  int G = want;
  while (G > 1 && base + (size_t)G * per > cap) G /= 2;
  return G;
}

mbinv_status run_group_psc(mbinv_ctx* c, const std::vector<Req>& reqs, mbinv_report* rep) {
  if (reqs.empty()) return MBINV_OK;
  if (c->l > 0 || c->hM || c->gen || c->opt.precision == MBINV_MIXED_BF16) return MBINV_ENOTSUP;
  const int G = (int)reqs.size();
  std::vector<const Schedule*> sch(G);
  for (int q = 0; q < G; ++q) sch[q] = psc_plan(c, reqs[q].i, reqs[q].j);
  if (c->opt.device_cap_bytes && base_bytes(c) + (size_t)G * sch[0]->planned > c->opt.device_cap_bytes)
    return MBINV_ENOMEM_CAP;
  release_sweep(c);
  const size_t planned = c->track.live + (size_t)G * sch[0]->planned;
  const int prec = c->opt.precision;
  const size_t sb = slot_bytes_for((int)c->b, prec);
  size_t per = 0;
  for (const Schedule* S : sch) per = std::max(per, (size_t)S->nslots * sb);
  CU(c->slots.ensure(per * G + 256));
  std::vector<Job> jobs(G);
  for (int q = 0; q < G; ++q) {
    Job& J = jobs[q];
    J.dM = c->dM;
    J.ldm = c->ldm;
    J.mdt = c->mdt;
    J.b = (int)c->b;
    J.slots = (char*)c->slots.p + per * q;
    J.slot_bytes = sb;
    J.slot_dt = env_slot_type(prec);
    J.out = reqs[q].dst;
    J.ldo = reqs[q].ldd;
    J.out_dt = c->odt;
    J.S = sch[q];
  }
  c->env.stream = c->stream;
  c->env.precision = prec;
  c->env.slices = c->opt.bf16_slices;
  c->env.profile = c->opt.profile != 0;
  c->env.inv_chunk = G;
  c->env.sing_tol = c->opt.sing_tol;
  c->env.pivot_cond = c->opt.pivot_cond != 0;
  c->env.use_graphs = c->opt.no_graphs == 0;
  const size_t replays0 = c->env.graph_replays;
  mbinv_status s = run_jobs(c->env, jobs);
  if (s == MBINV_ECUDA) last_cuda_error() = c->env.last_error;
  if (rep) {
    for (const Schedule* S : sch) add_report(rep, c, *S);
    rep->launches += (size_t)c->env.launches;
    rep->gemm_launches += (size_t)c->env.gemm_launches;
    add_env_report(rep, c->env);
    rep->planned_device_bytes = std::max(rep->planned_device_bytes, planned);
    rep->max_pivot_cond = std::max(rep->max_pivot_cond, c->env.max_cond);
    rep->graph_replays += c->env.graph_replays - replays0;
    if (s == MBINV_ESINGULAR && rep->failed_pivot < 0) rep->failed_pivot = c->env.failed_inverse;
  }
  return s;
}

// Runs any list of requests: groups of at most `width` with one border each.
mbinv_status run_requests(mbinv_ctx* c, const std::vector<Req>& reqs, int width, mbinv_report* rep) {
  std::map<int, std::vector<Req>> by_border;
  const bool psc = c->opt.variant == MBINV_VARIANT_PRINCIPAL && c->k >= 2;
  // the variant's diagonal and off-diagonal schedules have different shapes
  for (const Req& r : reqs) by_border[border_of(c, r.i, r.j) + (psc && r.i == r.j ? 8 : 0)].push_back(r);
  for (auto& kv : by_border) {
    const std::vector<Req>& v = kv.second;
    const int want = std::min<int>(std::max(1, width), (int)v.size());
    const int G = std::max(1, psc ? fit_group_psc(c, v, want) : fit_group(c, v, want));
    for (size_t q0 = 0; q0 < v.size(); q0 += G) {
      std::vector<Req> grp(v.begin() + q0, v.begin() + std::min(v.size(), q0 + G));
      mbinv_status s = psc ? run_group_psc(c, grp, rep) : run_group(c, grp, rep);
      if (s != MBINV_OK) return s;
    }
  }
  return MBINV_OK;
}

void start_report(mbinv_report* rep) {
  if (!rep) return;
  std::memset(rep, 0, sizeof *rep);
  rep->failed_pivot = -1;
}

// Blocks to caller buffers (host or device, any leading dimension, partial
// last blocks): full device blocks are written in place, the others go
// through the staging buffer one group at a time.
mbinv_status blocks_to(mbinv_ctx* c, const std::vector<std::pair<int64_t, int64_t>>& ij,
                       const std::vector<void*>& outs, const std::vector<int64_t>& ldos, int width,
                       mbinv_report* rep) {
  const size_t es = dtype_size(c->odt);
  std::vector<Req> direct;
  std::vector<size_t> staged;
  for (size_t t = 0; t < ij.size(); ++t) {
    const bool full = block_extent(c, ij[t].first) == c->b && block_extent(c, ij[t].second) == c->b;
    if (full && is_device_ptr(outs[t]))
      direct.push_back(Req{ij[t].first, ij[t].second, outs[t], ldos[t]});
    else
      staged.push_back(t);
  }
  mbinv_status s = run_requests(c, direct, width, rep);
  if (s != MBINV_OK) return s;
  if (staged.empty()) return MBINV_OK;
  const int W = std::max(1, std::min<int>(width, (int)staged.size()));
  CU(c->outtmp.ensure((size_t)W * c->b * c->b * 8 + 256));
  for (size_t q0 = 0; q0 < staged.size(); q0 += W) {
    std::vector<Req> grp;
    for (size_t u = q0; u < std::min(staged.size(), q0 + W); ++u)
      grp.push_back(Req{ij[staged[u]].first, ij[staged[u]].second,
                        (char*)c->outtmp.p + (u - q0) * (size_t)c->b * c->b * es, c->b});
    s = run_requests(c, grp, W, rep);
    if (s != MBINV_OK) return s;
    for (size_t u = q0; u < std::min(staged.size(), q0 + W); ++u) {
      const size_t t = staged[u];
      const int64_t bi = block_extent(c, ij[t].first), bj = block_extent(c, ij[t].second);
      const bool dev = is_device_ptr(outs[t]);
      CU(cudaMemcpy2DAsync(outs[t], (size_t)ldos[t] * es, (char*)c->outtmp.p + (u - q0) * (size_t)c->b * c->b * es,
                           (size_t)c->b * es, (size_t)bj * es, (size_t)bi,
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    }
    CU(cudaStreamSynchronize(c->stream));
  }
  return MBINV_OK;
}

constexpr int kDefaultWidth = 8;  // requests run together by default

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
  CU(c->gemmdesc.ensure(256));
  CU(cudaMemcpyAsync(c->gemmdesc.p, &d, sizeof d, cudaMemcpyHostToDevice, c->stream));
  CU(launch_gemm_grouped(combo, (const GemmDesc*)c->gemmdesc.p, 1, tiles, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return MBINV_OK;
}

mbinv_status row_or_col(mbinv_ctx* c, int64_t t, bool row, void* out, int64_t ldo, mbinv_report* rep) {
  std::vector<std::pair<int64_t, int64_t>> ij;
  std::vector<void*> outs;
  std::vector<int64_t> ldos;
  const size_t es = dtype_size(c->odt);
  for (int64_t q = 0; q < c->k; ++q) {
    ij.emplace_back(row ? t : q, row ? q : t);
    outs.push_back(row ? (char*)out + (size_t)q * c->b * es : (char*)out + (size_t)q * c->b * ldo * es);
    ldos.push_back(ldo);
  }
  return blocks_to(c, ij, outs, ldos, (int)c->k, rep);
}

// One two-sided refinement step (refined_blocks below), on any path:
//   X_i = block row i, Y_j = block column j of M^-1 from the sweep (kept in
//         FP32 on the FP32-valued paths, FP64 on FP64 and FP64_TC),
//   R   = E_i^T - X_i M                      (FP64 accumulation)
//   N_ij <- X_i E_j + R Y_j                  (FP64)
// With dX, dY the errors of X_i, Y_j the result differs from N_ij by
// -dX M dY: the error is squared when it is small.

// Uploads and runs a list of GEMM descriptors of one element-type combination.
mbinv_status gemm_list(mbinv_ctx* c, int combo, std::vector<GemmDesc>& ds) {
  if (ds.empty()) return MBINV_OK;
  int bm, bn, tiles = 0;
  gemm_tile_shape(combo, &bm, &bn);
  for (GemmDesc& d : ds) {
    d.tiles_n = (d.n + bn - 1) / bn;
    d.tile_start = tiles;
    tiles += ((d.m + bm - 1) / bm) * d.tiles_n;
  }
  CU(c->gemmdesc.ensure(ds.size() * sizeof(GemmDesc) + 256));
  CU(cudaMemcpyAsync(c->gemmdesc.p, ds.data(), ds.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice, c->stream));
  CU(launch_gemm_grouped(combo, (const GemmDesc*)c->gemmdesc.p, (int)ds.size(), tiles, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return MBINV_OK;
}

// C = beta Cin + alpha A B for every op (FP64, row-major; alpha +-1, beta 0 or
// 1; one inner length k for all) as FP64-accurate digit products on the
// tensor cores: each distinct A and B is packed once, then one grouped launch
// per K chunk of 512.  The sweep's digit buffers are reused: the sweep is over.
struct OzOp {
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  const double* cin;
  int64_t ldcin;
  double* C;
  int64_t ldc;
  int m, n;
  int ta = 0, tb = 0;  // A given as its transpose (k x m), B as its transpose (n x k)
};

mbinv_status oz_list(mbinv_ctx* c, const std::vector<OzOp>& ops, int k, double alpha, double beta) {
  if (ops.empty()) return MBINV_OK;
  auto up = [](size_t x, size_t q) { return (x + q - 1) / q * q; };
  std::map<const double*, int> aslab, bslab;
  std::vector<oz::PackDesc> pa, pb;
  int mmax = 1, nmax = 1;
  for (const OzOp& o : ops) {
    mmax = std::max(mmax, o.m);
    nmax = std::max(nmax, o.n);
    // slab rows are the rows of A and the columns of B
    if (aslab.emplace(o.A, (int)pa.size()).second)
      pa.push_back(o.ta ? oz::PackDesc{o.A, o.lda, k, o.m, 1, (int)pa.size()}
                        : oz::PackDesc{o.A, o.lda, o.m, k, 0, (int)pa.size()});
    if (bslab.emplace(o.B, (int)pb.size()).second)
      pb.push_back(o.tb ? oz::PackDesc{o.B, o.ldb, o.n, k, 0, (int)pb.size()}
                        : oz::PackDesc{o.B, o.ldb, k, o.n, 1, (int)pb.size()});
  }
  const int rpa = (int)up(mmax, oz::tile_m()), rpb = (int)up(nmax, oz::tile_n()), kpad = (int)up(k, oz::tile_k());
  const int nkb = kpad / oz::tile_k(), nchunk = (nkb + oz::kMaxKBlocks - 1) / oz::kMaxKBlocks;
  Env& E = c->env;
  CU(E.apk.ensure(pa.size() * (size_t)oz::kDigits * rpa * kpad * 2));
  CU(E.bpk.ensure(pb.size() * (size_t)oz::kDigits * rpb * kpad * 2));
  CU(E.oexp.ensure((pa.size() * rpa + pb.size() * rpb) * 4 + 256));
  CU(E.tcerr.ensure(256));
  int* ea = (int*)E.oexp.p;
  int* eb = ea + pa.size() * rpa;
  // descriptors: A packs, B packs, then the problems of every K chunk
  const size_t oa = 0, ob = up(pa.size() * sizeof(oz::PackDesc), 256),
               op = ob + up(pb.size() * sizeof(oz::PackDesc), 256), per = up(ops.size() * sizeof(oz::Problem), 256);
  std::vector<char> h(op + nchunk * per);
  std::memcpy(h.data() + oa, pa.data(), pa.size() * sizeof(oz::PackDesc));
  std::memcpy(h.data() + ob, pb.data(), pb.size() * sizeof(oz::PackDesc));
  for (int ch = 0; ch < nchunk; ++ch) {
    oz::Problem* pr = (oz::Problem*)(h.data() + op + ch * per);
    for (size_t t = 0; t < ops.size(); ++t) {
      const OzOp& o = ops[t];
      oz::Problem q{};
      q.a_slab = aslab[o.A];
      q.b_slab = bslab[o.B];
      q.cin = ch == 0 ? o.cin : o.C;  // later chunks add to what the first wrote
      q.ldcin = ch == 0 ? o.ldcin : o.ldc;
      q.out = o.C;
      q.ldo = o.ldc;
      q.m = o.m;
      q.n = o.n;
      pr[t] = q;
    }
  }
  CU(c->gemmdesc.ensure(h.size() + 256));
  char* d = (char*)c->gemmdesc.p;
  CU(cudaMemcpyAsync(d, h.data(), h.size(), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemsetAsync(E.tcerr.p, 0, sizeof(int), c->stream));
  CU(oz::launch_pack2(oz::PackSet{(const oz::PackDesc*)(d + oa), (int)pa.size(), rpa, (__nv_bfloat16*)E.apk.p, ea},
                      oz::PackSet{(const oz::PackDesc*)(d + ob), (int)pb.size(), rpb, (__nv_bfloat16*)E.bpk.p, eb},
                      kpad, c->stream));
  oz::Params Q{};
  Q.kpad = kpad;
  Q.tiles_m = rpa / oz::tile_m();
  Q.tiles_n = rpb / oz::tile_n();
  Q.alpha = alpha;
  Q.ea = ea;
  Q.eb = eb;
  Q.ea_rows = rpa;
  Q.eb_rows = rpb;
  Q.err = (int*)E.tcerr.p;
  for (int ch = 0; ch < nchunk; ++ch) {
    Q.kb0 = ch * oz::kMaxKBlocks;
    Q.nkb = std::min(oz::kMaxKBlocks, nkb - Q.kb0);
    Q.beta = ch == 0 ? beta : 1.0;
    CU(oz::launch_gemm((const __nv_bfloat16*)E.apk.p, (int)pa.size(), rpa, (const __nv_bfloat16*)E.bpk.p,
                       (int)pb.size(), rpb, Q, (const oz::Problem*)(d + op + ch * per), (int)ops.size(), c->stream));
  }
  int herr = 0;
  CU(cudaMemcpyAsync(&herr, E.tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return herr ? MBINV_ETIMEOUT : MBINV_OK;
}

GemmDesc gdesc(const void* A, int64_t lda, const void* B, int64_t ldb, const void* Cin, int64_t ldcin, void* C,
               int64_t ldc, int m, int n, int k, double alpha, double beta) {
  GemmDesc d{};
  d.A = A;
  d.lda = lda;
  d.B = B;
  d.ldb = ldb;
  d.Cin = Cin;
  d.ldcin = ldcin;
  d.C = C;
  d.ldc = ldc;
  d.m = m;
  d.n = n;
  d.k = k;
  d.alpha = alpha;
  d.beta = beta;
  return d;
}

// Refinement of many blocks at once: the block rows X_i and block columns Y_j
// they need are computed once (every block of them by its own run, width runs
// executed together), then one residual E_i^T - X_i M per distinct row and
// one correction X_i E_j + R_i Y_j per block, each set in one grouped launch.
mbinv_status refined_blocks(mbinv_ctx* c, const std::vector<std::pair<int64_t, int64_t>>& v,
                            const std::vector<void*>& outs, const std::vector<int64_t>& ldos, int width,
                            mbinv_report* rep) {
  const int64_t n = c->n, b = c->b, k = c->k;
  if (c->hM || c->gen) return MBINV_ENOTSUP;  // the residual reads all of M on the device
  std::map<int64_t, int> rows, cols;
  for (auto& p : v) {
    rows.emplace(p.first, (int)rows.size());
    cols.emplace(p.second, (int)cols.size());
  }
  // the sweeps' values in their own precision: FP64 on the FP64-valued paths
  const int xt = (c->opt.precision == MBINV_FP64 || c->opt.precision == MBINV_FP64_TC) ? F64 : F32;
  const size_t xs = dtype_size(xt);
  const size_t rsz = (size_t)b * n, csz = (size_t)n * b;
  CU(c->rowbuf.ensure(rows.size() * rsz * xs + 256));
  CU(c->colbuf.ensure(cols.size() * csz * xs + 256));
  char* X = (char*)c->rowbuf.p;  // X_i at X + (rows[i] * rsz) * xs, leading dimension n
  char* Y = (char*)c->colbuf.p;  // Y_j at Y + (cols[j] * csz) * xs, leading dimension b
  // every block of the needed rows and columns, each computed once
  std::vector<std::pair<int64_t, int64_t>> ij;
  std::vector<void*> dst;
  std::vector<int64_t> ld;
  std::vector<std::pair<int64_t, int64_t>> copies;  // blocks also needed in a column
  for (auto& r : rows)
    for (int64_t q = 0; q < k; ++q) {
      ij.emplace_back(r.first, q);
      dst.push_back(X + (r.second * rsz + q * b) * xs);
      ld.push_back(n);
      if (cols.count(q)) copies.emplace_back(r.first, q);
    }
  for (auto& cc : cols)
    for (int64_t q = 0; q < k; ++q) {
      if (rows.count(q)) continue;
      ij.emplace_back(q, cc.first);
      dst.push_back(Y + (cc.second * csz + q * b * b) * xs);
      ld.push_back(b);
    }
  const int saved_dtype = c->odt;
  c->odt = xt;  // the sweeps write blocks in the working type
  mbinv_status s = blocks_to(c, ij, dst, ld, width, rep);
  c->odt = saved_dtype;
  if (s != MBINV_OK) return s;
  for (auto& p : copies) {
    const int64_t bi = block_extent(c, p.first), bj = block_extent(c, p.second);
    CU(cudaMemcpy2DAsync(Y + (cols[p.second] * csz + p.first * b * b) * xs, (size_t)b * xs,
                         X + (rows[p.first] * rsz + p.second * b) * xs, (size_t)n * xs, (size_t)bj * xs, (size_t)bi,
                         cudaMemcpyDeviceToDevice, c->stream));
  }
  // R_i = -X_i M + E_i^T (FP64_TC: as digit products on the tensor cores);
  // under a cap the sweep's workspace goes first
  release_sweep(c);
  CU(c->resid.ensure(rows.size() * rsz * 8 + v.size() * (size_t)b * b * 8 + 512));
  double* R = (double*)c->resid.p;
  double* Nb = R + rows.size() * rsz;
  const bool tcr = c->opt.precision == MBINV_FP64_TC && c->mdt == F64;
  std::vector<GemmDesc> ds;
  std::vector<OzOp> zs;
  for (auto& r : rows) {
    ds.push_back(gdesc(X + r.second * rsz * xs, n, c->dM, c->ldm, nullptr, 0, R + r.second * rsz, n,
                       (int)block_extent(c, r.first), (int)n, (int)n, -1.0, 0.0));
    zs.push_back(OzOp{(const double*)(X + r.second * rsz * xs), n, (const double*)c->dM, c->ldm, nullptr, 0,
                      R + r.second * rsz, n, (int)block_extent(c, r.first), (int)n});
  }
  s = tcr ? oz_list(c, zs, (int)n, -1.0, 0.0)
          : gemm_list(c, xt == F64 ? G_F64 : (c->mdt == F64 ? G_F32F64_F64 : G_F32IN_F64), ds);
  if (s != MBINV_OK) return s;
  double rmax = 0;
  for (auto& r : rows) {
    const int64_t bi = block_extent(c, r.first);
    double* Ri = R + r.second * rsz;
    add_eye_kernel<<<(unsigned)((bi + 255) / 256), 256, 0, c->stream>>>(Ri, n, r.first * b, bi);
    CU(cudaGetLastError());
    double* acc = Nb + v.size() * (size_t)b * b;
    CU(cudaMemsetAsync(acc, 0, sizeof(double), c->stream));
    sumsq_kernel<<<64, 256, 0, c->stream>>>(Ri, n, bi, n, acc);
    CU(cudaGetLastError());
    double h = 0;
    CU(cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    rmax = std::max(rmax, std::sqrt(h / (double)bi));
  }
  // N_ij = X_i E_j + R_i Y_j
  ds.clear();
  zs.clear();
  for (size_t t = 0; t < v.size(); ++t) {
    const int64_t i = v[t].first, j = v[t].second;
    const int64_t bi = block_extent(c, i), bj = block_extent(c, j);
    double* Nt = Nb + t * (size_t)b * b;
    const char* Xij = X + (rows[i] * rsz + j * b) * xs;
    if (xt == F64)
      convert_kernel<double, double><<<(unsigned)((bi * bj + 255) / 256), 256, 0, c->stream>>>(
          (const double*)Xij, n, Nt, bj, bi, bj);
    else
      convert_kernel<float, double><<<(unsigned)((bi * bj + 255) / 256), 256, 0, c->stream>>>(
          (const float*)Xij, n, Nt, bj, bi, bj);
    CU(cudaGetLastError());
    ds.push_back(gdesc(R + rows[i] * rsz, n, Y + cols[j] * csz * xs, b, Nt, bj, Nt, bj, (int)bi, (int)bj, (int)n,
                       1.0, 1.0));
    zs.push_back(OzOp{R + rows[i] * rsz, n, (const double*)(Y + cols[j] * csz * xs), b, Nt, bj, Nt, bj, (int)bi,
                      (int)bj});
  }
  s = tcr ? oz_list(c, zs, (int)n, 1.0, 1.0) : gemm_list(c, xt == F64 ? G_F64 : G_F64F32_F64, ds);
  if (s != MBINV_OK) return s;
  const size_t es = dtype_size(c->odt);
  for (size_t t = 0; t < v.size(); ++t) {
    const int64_t bi = block_extent(c, v[t].first), bj = block_extent(c, v[t].second);
    double* Nt = Nb + t * (size_t)b * b;
    const bool dev = is_device_ptr(outs[t]);
    if (c->odt == F64) {
      CU(cudaMemcpy2DAsync(outs[t], (size_t)ldos[t] * es, Nt, (size_t)bj * 8, (size_t)bj * 8, (size_t)bi,
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    } else {
      CU(c->outtmp.ensure((size_t)b * b * 8 + 256));
      convert_kernel<double, float><<<(unsigned)((bi * bj + 255) / 256), 256, 0, c->stream>>>(
          Nt, bj, (float*)c->outtmp.p, bj, bi, bj);
      CU(cudaGetLastError());
      CU(cudaMemcpy2DAsync(outs[t], (size_t)ldos[t] * es, c->outtmp.p, (size_t)bj * 4, (size_t)bj * 4, (size_t)bi,
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
      CU(cudaStreamSynchronize(c->stream));
    }
  }
  CU(cudaStreamSynchronize(c->stream));
  if (rep) {
    for (auto& r : rows) rep->gemm_flops += 2.0 * block_extent(c, r.first) * n * n;
    for (auto& p : v) rep->gemm_flops += 2.0 * block_extent(c, p.first) * block_extent(c, p.second) * n;
    rep->launches += 2 + 2 * rows.size() + v.size();
    rep->rel_residual = std::max(rep->rel_residual, rmax);

  }
  if (!(rmax < 1.0)) return MBINV_ENOTCONV;
  return MBINV_OK;
}

}  // namespace

// Synthetic matrices of the autotuner: uniform[-1, 1) (a SplitMix64 hash of
// the element index) plus b on the diagonal.
__global__ void tune_fill_kernel(double* a, int64_t count, int64_t b) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count * b * b) return;
  const uint64_t u = sm64_mix(sm64_mix(0x7475ull) + (uint64_t)(e + 1) * 0x9E3779B97F4A7C15ull);
  double v = 2.0 * ((double)(u >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
  const int64_t r = (e / b) % b, c = e % b;
  if (r == c) v += (double)b;
  a[e] = v;
}

// Applies the lines "b count precision bias seconds" of a cache file.
void load_tune_cache(const char* path) {
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  long long b, count;
  int prec, bias;
  double secs;
  while (fscanf(f, "%lld %lld %d %d %lf", &b, &count, &prec, &bias, &secs) == 5)
    if (b > 0 && count > 0 && prec >= MBINV_FP64 && prec <= MBINV_FP64_TC && bias >= -3 && bias <= 3)
      set_cluster_bias((int)b, (int)count, env_work_type(prec), prec == MBINV_FP64_TC, bias);
  fclose(f);
}

// Nothing may be thrown across the C ABI: a failed host allocation or any
// other exception inside a call becomes a status.
template <typename F>
mbinv_status guarded(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return MBINV_ENOMEM_CAP;
  } catch (...) {
    return MBINV_EINVAL;
  }
}

// One call on a context: under a cap the context first lets go of the
// workspace an earlier call left (buffers only grow within a call), and the
// report carries the measured high-water mark of the call.  The nested calls
// some entry points make (mbinv_all_blocks runs mbinv_blocks) keep the
// outermost call's mark.
template <typename F>
mbinv_status on_context(mbinv_ctx* c, mbinv_report* rep, F&& f) {
  if (!c) return MBINV_EINVAL;
  const bool outer = c->depth++ == 0;
  if (outer) {
    if (c->opt.device_cap_bytes) {
      if (c->stream) cudaStreamSynchronize(c->stream);
      for (DevBuf* d : c->bufs())
        if (d != &c->own_M) d->release();
    }
    c->track.hwm = c->track.live;
  }
  mbinv_status s = guarded(f);
  --c->depth;
  if (rep) rep->peak_device_bytes = std::max(rep->peak_device_bytes, c->track.hwm);
  return s;
}

// ====================================================================== ABI

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
    case MBINV_ECALLBACK: return "the matrix producer failed";
  }
  return "unknown status";
}

const char* mbinv_version(void) { return "mbinv 0.2 (sm_103a)"; }

const char* mbinv_last_cuda_error(void) { return cudaGetErrorString(last_cuda_error()); }

// Copies the caller's M (c->srcM) into the context's own device matrix,
// converting it to the sweep's element type where they differ, and writes the
// padded corner (identity) and border strips.  On c->stream; returns once the
// copy is complete (the caller may then change its buffer).
static mbinv_status upload_m(mbinv_ctx* c, MemTrack* tr) {
  const int64_t n = c->n;
  const int dtype = c->dtype;
  const size_t es = dtype_size(dtype), mes = dtype_size(c->mdt);
  const void* M = c->srcM;
  const int64_t ld = c->srcld;
  const bool dev = c->srcdev;
  if (c->mdt == dtype) {
    CU(cudaMemcpy2DAsync(c->own_M.p, (size_t)c->npad * mes, M, (size_t)ld * es, (size_t)n * es, (size_t)n,
                         dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  } else {
    // stage the caller's matrix on the device, then convert it
    DevBuf stage;
    stage.track = tr;
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
    c->border_mode = -1;
    mbinv_status s = set_border(c, 0);
    if (s != MBINV_OK) return s;
  }
  CU(cudaStreamSynchronize(c->stream));
  return MBINV_OK;
}

// shared: the tracker of a batched call, whose contexts count their bytes
// together (no cap of their own); null for an ordinary context.
static mbinv_status mbinv_create_impl(mbinv_ctx** out, int64_t n, int64_t k, int dtype, const void* M, int64_t ld,
                                      const mbinv_options* opt, MemTrack* shared = nullptr) {
  if (!out || !M || n <= 0 || k <= 0 || k > 63 || k > n || ld < n || (dtype != F64 && dtype != F32))
    return MBINV_EINVAL;
  *out = nullptr;
  mbinv_options o;
  mbinv_default_options(&o);
  if (opt) {
    if (opt->struct_size != sizeof(mbinv_options)) return MBINV_EINVAL;
    o = *opt;
  }
  if (o.precision < MBINV_FP64 || o.precision > MBINV_FP64_TC) return MBINV_EINVAL;
  if (o.precision == MBINV_MIXED_BF16 && (o.bf16_slices < 1 || o.bf16_slices > 3)) return MBINV_EINVAL;
  if (o.refine_steps < 0 || o.refine_steps > 1) return MBINV_EINVAL;
  if (o.out_dtype < 0 || o.out_dtype > 2 || o.schedule < 0 || o.schedule > 2 || !(o.sing_tol >= 0.0) ||
      o.variant < 0 || o.variant > 1)
    return MBINV_EINVAL;
  std::unique_ptr<mbinv_ctx> c(new (std::nothrow) mbinv_ctx);
  if (!c) return MBINV_EINVAL;
  c->n = n;
  c->k = k;
  c->b = (n + k - 1) / k;
  c->npad = c->b * k;
  c->l = c->npad - n;
  c->dtype = dtype;
  c->odt = o.out_dtype == 1 ? F64 : (o.out_dtype == 2 ? F32 : dtype);
  c->opt = o;
  load_tune_cache(o.tune_cache_path);
  c->track.cap = shared ? 0 : o.device_cap_bytes;
  MemTrack* tr = shared ? shared : &c->track;
  for (DevBuf* d : c->bufs()) d->track = tr;
  c->stream = (cudaStream_t)o.cuda_stream;
  // the plain paths read M in their own precision; the mixed path reads the
  // caller's M as given (its residual is taken against it)
  c->mdt = (o.precision == MBINV_FP64 || o.precision == MBINV_FP64_TC) ? F64
                                                                          : (o.precision == MBINV_FP32 ? F32 : dtype);
  const size_t es = dtype_size(dtype), mes = dtype_size(c->mdt);
  const bool dev = is_device_ptr(M);
  const size_t mbytes_dev = (size_t)c->npad * c->npad * mes;
  const size_t slot16 = 16 * slot_bytes_for((int)c->b, o.precision);
  if (!dev && !shared && c->l == 0 && k >= 2 && o.precision != MBINV_MIXED_BF16 &&
      o.schedule != MBINV_SCHEDULE_LEVELS &&
      (o.schedule == MBINV_SCHEDULE_BOUNDED || (o.device_cap_bytes && mbytes_dev + slot16 > o.device_cap_bytes))) {
    // M stays in host memory, read block by block by the bounded schedule
    c->hM = M;
    c->hld = ld;
    *out = c.release();
    return MBINV_OK;
  }
  if (c->l == 0 && dev && c->mdt == dtype) {
    c->dM = M;
    c->ldm = ld;
  } else {
    const size_t mbytes = (size_t)c->npad * c->npad * mes;
    if (o.device_cap_bytes && mbytes > o.device_cap_bytes) return MBINV_ENOMEM_CAP;
    CU(c->own_M.ensure(mbytes));
    c->dM = c->own_M.p;
    c->ldm = c->npad;
    c->srcM = M;
    c->srcld = ld;
    c->srcdev = dev;
    mbinv_status s = upload_m(c.get(), tr);
    if (s != MBINV_OK) return s;
    CU(cudaStreamSynchronize(c->stream));
  }
  *out = c.release();
  return MBINV_OK;
}

static mbinv_status mbinv_create_from_fn_impl(mbinv_ctx** out, int64_t n, int64_t k, int dtype, mbinv_block_fn fn,
                                              void* user, const mbinv_options* opt) {
  if (!out || !fn || n <= 0 || k < 2 || k > 63 || k > n || (dtype != F64 && dtype != F32)) return MBINV_EINVAL;
  *out = nullptr;
  mbinv_options o;
  mbinv_default_options(&o);
  if (opt) {
    if (opt->struct_size != sizeof(mbinv_options)) return MBINV_EINVAL;
    o = *opt;
  }
  if (o.precision < MBINV_FP64 || o.precision > MBINV_FP64_TC || o.refine_steps < 0 || o.refine_steps > 1 ||
      o.out_dtype < 0 || o.out_dtype > 2 || o.schedule < 0 || o.schedule > 2 || !(o.sing_tol >= 0.0))
    return MBINV_EINVAL;
  if (n % k || o.precision == MBINV_MIXED_BF16 || o.refine_steps || o.schedule == MBINV_SCHEDULE_LEVELS)
    return MBINV_ENOTSUP;
  std::unique_ptr<mbinv_ctx> c(new (std::nothrow) mbinv_ctx);
  if (!c) return MBINV_EINVAL;
  c->n = n;
  c->k = k;
  c->b = n / k;
  c->npad = n;
  c->l = 0;
  c->dtype = dtype;
  c->odt = o.out_dtype == 1 ? F64 : (o.out_dtype == 2 ? F32 : dtype);
  c->opt = o;
  load_tune_cache(o.tune_cache_path);
  c->track.cap = o.device_cap_bytes;
  for (DevBuf* d : c->bufs()) d->track = &c->track;
  c->stream = (cudaStream_t)o.cuda_stream;
  c->mdt = (o.precision == MBINV_FP64 || o.precision == MBINV_FP64_TC) ? F64 : F32;
  c->gen = fn;
  c->gen_user = user;
  *out = c.release();
  return MBINV_OK;
}

void mbinv_destroy(mbinv_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (DevBuf* d : {&c->own_M, &c->slots, &c->outtmp, &c->rowbuf, &c->colbuf, &c->resid, &c->gbuf, &c->wbuf,
                    &c->dmbuf, &c->gemmdesc})
    d->release();
  c->env.release();
  c->spill.release();
  delete c;
}

static mbinv_status mbinv_block_impl(mbinv_ctx* c, int64_t i, int64_t j, void* out, int64_t ldo, mbinv_report* rep) {
  if (!c || !out || i < 0 || j < 0 || i >= c->k || j >= c->k) return MBINV_EINVAL;
  if (ldo < block_extent(c, j)) return MBINV_EINVAL;
  start_report(rep);
  auto t0 = std::chrono::steady_clock::now();
  mbinv_status s;
  if (c->opt.refine_steps > 0 && !c->in_sweep) {
    c->in_sweep = true;
    s = refined_blocks(c, {{i, j}}, {out}, {ldo}, kDefaultWidth, rep);
    c->in_sweep = false;
  } else {
    s = blocks_to(c, {{i, j}}, {out}, {ldo}, 1, rep);
  }
  if (rep) rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

static mbinv_status mbinv_blocks_impl(mbinv_ctx* c, int64_t count, const int64_t* ij, void* const* outs, const int64_t* ldos,
                          int width, mbinv_report* rep) {
  if (!c || count < 0 || (count > 0 && (!ij || !outs || !ldos))) return MBINV_EINVAL;
  std::vector<std::pair<int64_t, int64_t>> v;
  std::vector<void*> o;
  std::vector<int64_t> l;
  for (int64_t t = 0; t < count; ++t) {
    const int64_t i = ij[2 * t], j = ij[2 * t + 1];
    if (i < 0 || j < 0 || i >= c->k || j >= c->k || !outs[t] || ldos[t] < block_extent(c, j)) return MBINV_EINVAL;
    v.emplace_back(i, j);
    o.push_back(outs[t]);
    l.push_back(ldos[t]);
  }
  start_report(rep);
  auto t0 = std::chrono::steady_clock::now();
  mbinv_status s = MBINV_OK;
  if (c->opt.refine_steps > 0) {
    c->in_sweep = true;
    s = refined_blocks(c, v, o, l, width > 0 ? width : kDefaultWidth, rep);
    c->in_sweep = false;
  } else {
    s = blocks_to(c, v, o, l, width > 0 ? width : kDefaultWidth, rep);
  }
  if (rep) rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

static mbinv_status mbinv_all_blocks_impl(mbinv_ctx* c, void* out, int64_t ldo, const uint8_t* done,
                                          mbinv_block_done_cb cb, void* user, mbinv_report* rep) {
  if (!c || !out || ldo < c->n) return MBINV_EINVAL;
  start_report(rep);
  auto t0 = std::chrono::steady_clock::now();
  const size_t es = dtype_size(c->odt);
  // the blocks still to do, in row-major order
  std::vector<std::pair<int64_t, int64_t>> todo;
  for (int64_t i = 0; i < c->k; ++i)
    for (int64_t j = 0; j < c->k; ++j)
      if (!(done && done[i * c->k + j])) todo.emplace_back(i, j);
  // Without a cap all runs go in one call, their shared frames evaluated once;
  // under a cap one block row at a time (mbinv_blocks splits further if the
  // cap asks).  The callback follows each finished chunk.
  const size_t chunk = c->opt.device_cap_bytes ? (size_t)c->k : todo.size();
  for (size_t q0 = 0; q0 < todo.size(); q0 += chunk) {
    const size_t q1 = std::min(todo.size(), q0 + chunk);
    std::vector<int64_t> ij;
    std::vector<void*> outs;
    std::vector<int64_t> ldos;
    for (size_t q = q0; q < q1; ++q) {
      const int64_t i = todo[q].first, j = todo[q].second;
      ij.push_back(i);
      ij.push_back(j);
      outs.push_back((char*)out + ((size_t)i * c->b * ldo + (size_t)j * c->b) * es);
      ldos.push_back(ldo);
    }
    mbinv_report r;
    mbinv_status s =
        mbinv_blocks(c, (int64_t)outs.size(), ij.data(), outs.data(), ldos.data(), (int)outs.size(), &r);
    if (rep) {
      rep->gemm_flops += r.gemm_flops;
      rep->inv_flops += r.inv_flops;
      rep->frames += r.frames;
      rep->request_frames += r.request_frames;
      rep->inversions += r.inversions;
      rep->launches += r.launches;
      rep->gemm_launches += r.gemm_launches;
      rep->gemm_device_seconds += r.gemm_device_seconds;
      rep->inv_device_seconds += r.inv_device_seconds;
      rep->pack_device_seconds += r.pack_device_seconds;
      rep->pack_bytes += r.pack_bytes;
      rep->inv_panel_device_seconds += r.inv_panel_device_seconds;
      rep->inv_panel_flops += r.inv_panel_flops;
      rep->inv_update_flops += r.inv_update_flops;
      rep->inv_panel_launches += r.inv_panel_launches;
      rep->rel_residual = std::max(rep->rel_residual, r.rel_residual);
      rep->max_pivot_cond = std::max(rep->max_pivot_cond, r.max_pivot_cond);
      rep->graph_replays += r.graph_replays;
      rep->host_in_bytes += r.host_in_bytes;
      rep->host_out_bytes += r.host_out_bytes;
      rep->host_spill_bytes = std::max(rep->host_spill_bytes, r.host_spill_bytes);
      rep->peak_device_bytes = std::max(rep->peak_device_bytes, r.peak_device_bytes);
      rep->planned_device_bytes = std::max(rep->planned_device_bytes, r.planned_device_bytes);
      if (s == MBINV_ESINGULAR) rep->failed_pivot = r.failed_pivot;
    }
    if (s != MBINV_OK) return s;
    if (cb)
      for (size_t q = q0; q < q1; ++q) cb(todo[q].first, todo[q].second, user);
  }
  if (rep) rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return MBINV_OK;
}

static mbinv_status mbinv_block_row_impl(mbinv_ctx* c, int64_t i, void* out, int64_t ldo, mbinv_report* rep) {
  if (!c || !out || i < 0 || i >= c->k || ldo < c->n) return MBINV_EINVAL;
  start_report(rep);
  return row_or_col(c, i, true, out, ldo, rep);
}

static mbinv_status mbinv_block_col_impl(mbinv_ctx* c, int64_t j, void* out, int64_t ldo, mbinv_report* rep) {
  if (!c || !out || j < 0 || j >= c->k || ldo < block_extent(c, j)) return MBINV_EINVAL;
  start_report(rep);
  return row_or_col(c, j, false, out, ldo, rep);
}

// One FP64 product C = beta Cin + alpha op(A) op(B) (op = transpose when ta /
// tb), as a digit product on the tensor cores on FP64_TC, else on the FP64
// CUDA-core GEMM.
mbinv_status prod64(mbinv_ctx* c, const double* A, int64_t lda, int ta, const double* B, int64_t ldb, int tb,
                    const double* Cin, int64_t ldcin, double* C, int64_t ldc, int m, int n, int k, double alpha,
                    double beta) {
  if (c->opt.precision == MBINV_FP64_TC) {
    OzOp o{A, lda, B, ldb, Cin, ldcin, C, ldc, m, n};
    o.ta = ta;
    o.tb = tb;
    return oz_list(c, {o}, k, alpha, Cin ? beta : 0.0);
  }
  return gemm1(c, G_F64, A, lda, ta, B, ldb, tb, Cin, ldcin, C, ldc, m, n, k, alpha, Cin ? beta : 0.0);
}

// The adjoint of L = sum(G .* N_ij): dM += -(X_i)^T G (Y_j)^T.  On the
// FP64-valued paths with refine_steps = 1 the whole approximate inverse N~
// (every block by the merged sweep) is first improved by Newton-Schulz steps
// N~ <- N~ + N~ (I - M N~) - each squares ||I - M N~|| - and X_i, Y_j are its
// block row and column.
static mbinv_status backward_fp64(mbinv_ctx* c, int64_t i, int64_t j, const void* G, int64_t ldg, void* dM,
                                  int64_t ldd, mbinv_report* rep) {
  const int64_t bi = block_extent(c, i), bj = block_extent(c, j), n = c->n, b = c->b;
  const bool refine = c->opt.refine_steps > 0;
  if (refine && (c->hM || c->gen || c->mdt != F64 || c->l > 0)) return MBINV_ENOTSUP;
  const size_t es = dtype_size(c->dtype);
  double *X, *Y;
  int64_t ldx, ldy;
  const int saved_odt = c->odt;
  c->odt = F64;  // rows, columns and the whole inverse come out in FP64
  mbinv_status s = MBINV_OK;
  if (refine) {
    // N~: all k^2 blocks, their runs merged (the all-blocks sweep of Sec. 5)
    CU(c->dmbuf.ensure((size_t)n * n * 8 + 256));
    std::vector<std::pair<int64_t, int64_t>> ij;
    std::vector<void*> outs;
    std::vector<int64_t> lds;
    for (int64_t r = 0; r < c->k; ++r)
      for (int64_t q = 0; q < c->k; ++q) {
        ij.emplace_back(r, q);
        outs.push_back((double*)c->dmbuf.p + (size_t)r * b * n + (size_t)q * b);
        lds.push_back(n);
      }
    s = blocks_to(c, ij, outs, lds, (int)ij.size(), rep);
    c->odt = saved_odt;
    if (s != MBINV_OK) return s;
    release_sweep(c);
    // Newton-Schulz on the whole approximate inverse: E = I - M N~,
    // N~ <- N~ + N~ E, which squares ||E|| each time (it converges when
    // ||E|| < 1); until ||E||_F / sqrt(n) stops falling - the last better N~
    // is kept - or is at the rounding level (at most 12 steps)
    CU(c->rowbuf.ensure((size_t)n * n * 8 + 256));
    CU(c->colbuf.ensure((size_t)n * n * 8 + 256));
    CU(c->resid.ensure(512));
    double* Nt = (double*)c->dmbuf.p;
    double* E = (double*)c->rowbuf.p;
    double* Nn = (double*)c->colbuf.p;
    double* acc = (double*)c->resid.p;
    double last = 1e300;
    for (int it = 0; it < 12; ++it) {
      s = prod64(c, (const double*)c->dM, c->ldm, 0, Nt, n, 0, nullptr, 0, E, n, (int)n, (int)n, (int)n, -1.0, 0.0);
      if (s != MBINV_OK) return s;
      add_eye_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(E, n, 0, n);
      CU(cudaGetLastError());
      CU(cudaMemsetAsync(acc, 0, sizeof(double), c->stream));
      sumsq_kernel<<<152, 256, 0, c->stream>>>(E, n, n, n, acc);
      CU(cudaGetLastError());
      double h = 0;
      CU(cudaMemcpyAsync(&h, acc, sizeof h, cudaMemcpyDeviceToHost, c->stream));
      CU(cudaStreamSynchronize(c->stream));
      const double res = std::sqrt(h / (double)n);
      if (rep) {
        rep->rel_residual = res;
        rep->gemm_flops += 2.0 * (double)n * n * n;
      }
      if (getenv("MBINV_TRACE_NS")) fprintf(stderr, "newton-schulz %d residual %.3e\n", it, res);
      if (!(res < last)) {  // no longer contracting: keep the previous, better N~
        if (it > 0) std::swap(Nt, Nn);
        if (rep) rep->rel_residual = last;
        break;
      }
      if (res < 1e-14) break;
      last = res;
      s = prod64(c, Nt, n, 0, E, n, 0, Nt, n, Nn, n, (int)n, (int)n, (int)n, 1.0, 1.0);
      if (s != MBINV_OK) return s;
      if (rep) rep->gemm_flops += 2.0 * (double)n * n * n;
      std::swap(Nt, Nn);
    }
    X = Nt + (size_t)i * b * n;
    ldx = n;
    Y = Nt + (size_t)j * b;
    ldy = n;
  } else {
    CU(c->rowbuf.ensure((size_t)b * n * 8 + 256));
    CU(c->colbuf.ensure((size_t)n * b * 8 + 256));
    s = row_or_col(c, i, true, c->rowbuf.p, n, rep);
    if (s == MBINV_OK) s = row_or_col(c, j, false, c->colbuf.p, bj, rep);
    c->odt = saved_odt;
    if (s != MBINV_OK) return s;
    X = (double*)c->rowbuf.p;
    ldx = n;
    Y = (double*)c->colbuf.p;
    ldy = bj;
  }
  // G and dM in FP64 on the device
  CU(c->gbuf.ensure((size_t)bi * bj * 8 + 256));
  double* Gd = (double*)c->gbuf.p;
  const bool gdev = is_device_ptr(G);
  if (c->dtype == F64) {
    CU(cudaMemcpy2DAsync(Gd, (size_t)bj * 8, G, (size_t)ldg * 8, (size_t)bj * 8, (size_t)bi,
                         gdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  } else {
    CU(c->outtmp.ensure((size_t)bi * bj * 4 + 256));
    CU(cudaMemcpy2DAsync(c->outtmp.p, (size_t)bj * 4, G, (size_t)ldg * 4, (size_t)bj * 4, (size_t)bi,
                         gdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    convert_kernel<float, double><<<(unsigned)((bi * bj + 255) / 256), 256, 0, c->stream>>>(
        (const float*)c->outtmp.p, bj, Gd, bj, bi, bj);
    CU(cudaGetLastError());
  }
  const bool dm_dev = is_device_ptr(dM);
  double* Dd;
  int64_t lddd;
  if (c->dtype == F64 && dm_dev) {
    Dd = (double*)dM;
    lddd = ldd;
  } else {
    CU(c->wbuf.ensure((size_t)n * n * 8 + (size_t)bi * n * 8 + 256));
    Dd = (double*)c->wbuf.p + (size_t)bi * n;
    lddd = n;
    if (c->dtype == F64) {
      CU(cudaMemcpy2DAsync(Dd, (size_t)n * 8, dM, (size_t)ldd * 8, (size_t)n * 8, (size_t)n, cudaMemcpyHostToDevice,
                           c->stream));
    } else {
      // FP32 dM: stage it (host or device), widen, accumulate in FP64, narrow back
      CU(c->outtmp.ensure((size_t)n * n * 4 + 256));
      CU(cudaMemcpy2DAsync(c->outtmp.p, (size_t)n * 4, dM, (size_t)ldd * 4, (size_t)n * 4, (size_t)n,
                           dm_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
      convert_kernel<float, double><<<(unsigned)((n * n + 255) / 256), 256, 0, c->stream>>>(
          (const float*)c->outtmp.p, n, Dd, n, n, n);
      CU(cudaGetLastError());
    }
  }
  CU(c->wbuf.ensure(std::max(c->wbuf.bytes, (size_t)bi * n * 8 + 256)));
  double* W = (double*)c->wbuf.p;
  // W = G Y_j^T (bi x n), then dM += -X_i^T W
  s = prod64(c, Gd, bj, 0, Y, ldy, 1, nullptr, 0, W, n, (int)bi, (int)n, (int)bj, 1.0, 0.0);
  if (s != MBINV_OK) return s;
  s = prod64(c, X, ldx, 1, W, n, 0, Dd, lddd, Dd, lddd, (int)n, (int)n, (int)bi, -1.0, 1.0);
  if (s != MBINV_OK) return s;
  if (!(c->dtype == F64 && dm_dev)) {
    if (c->dtype == F64) {
      CU(cudaMemcpy2DAsync(dM, (size_t)ldd * 8, Dd, (size_t)n * 8, (size_t)n * 8, (size_t)n, cudaMemcpyDeviceToHost,
                           c->stream));
    } else {
      convert_kernel<double, float><<<(unsigned)((n * n + 255) / 256), 256, 0, c->stream>>>(
          Dd, n, (float*)c->outtmp.p, n, n, n);
      CU(cudaGetLastError());
      CU(cudaMemcpy2DAsync(dM, (size_t)ldd * 4, c->outtmp.p, (size_t)n * 4, (size_t)n * 4, (size_t)n,
                           dm_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    }
  }
  CU(cudaStreamSynchronize(c->stream));
  if (rep) {
    rep->gemm_flops += 2.0 * bi * bj * n + 2.0 * n * n * bi;
    rep->launches += 2;
  }
  (void)es;
  return MBINV_OK;
}

static mbinv_status backward_same_type(mbinv_ctx* c, int64_t i, int64_t j, const void* G, int64_t ldg, void* dM, int64_t ldd,
                            mbinv_report* rep) {
  const int64_t bi = block_extent(c, i), bj = block_extent(c, j), n = c->n;
  const size_t es = dtype_size(c->dtype);
  const int combo = c->dtype == F64 ? G_F64 : G_F32;
  // X_i (bi x n) and Y_j (n x bj) of M^-1, their blocks run together
  CU(c->rowbuf.ensure((size_t)c->b * n * es + 256));
  CU(c->colbuf.ensure((size_t)n * c->b * es + 256));
  // the rows and columns come out in M's type, the type of G and dM
  const int saved_odt = c->odt;
  c->odt = c->dtype;
  mbinv_status s = row_or_col(c, i, true, c->rowbuf.p, n, rep);
  if (s == MBINV_OK) s = row_or_col(c, j, false, c->colbuf.p, bj, rep);
  c->odt = saved_odt;
  if (s != MBINV_OK) return s;
  const void* Gd = G;
  if (!is_device_ptr(G)) {
    CU(c->gbuf.ensure((size_t)bi * bj * es));
    CU(cudaMemcpy2DAsync(c->gbuf.p, (size_t)bj * es, G, (size_t)ldg * es, (size_t)bj * es, (size_t)bi,
                         cudaMemcpyHostToDevice, c->stream));
    Gd = c->gbuf.p;
    ldg = bj;
  }
  void* Dd = dM;
  int64_t lddd = ldd;
  const bool dm_host = !is_device_ptr(dM);
  if (dm_host) {
    CU(c->dmbuf.ensure((size_t)n * n * es));
    CU(cudaMemcpy2DAsync(c->dmbuf.p, (size_t)n * es, dM, (size_t)ldd * es, (size_t)n * es, (size_t)n,
                         cudaMemcpyHostToDevice, c->stream));
    Dd = c->dmbuf.p;
    lddd = n;
  }
  // W = G Y_j^T (bi x n), then dM += -X_i^T W
  CU(c->wbuf.ensure((size_t)bi * n * es));
  s = gemm1(c, combo, Gd, ldg, 0, c->colbuf.p, bj, 1, nullptr, 0, c->wbuf.p, n, (int)bi, (int)n, (int)bj, 1.0, 0.0);
  if (s != MBINV_OK) return s;
  s = gemm1(c, combo, c->rowbuf.p, n, 1, c->wbuf.p, n, 0, Dd, lddd, Dd, lddd, (int)n, (int)n, (int)bi, -1.0, 1.0);
  if (s != MBINV_OK) return s;
  if (dm_host) {
    CU(cudaMemcpy2DAsync(dM, (size_t)ldd * es, c->dmbuf.p, (size_t)n * es, (size_t)n * es, (size_t)n,
                         cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  if (rep) {
    rep->gemm_flops += 2.0 * bi * bj * n + 2.0 * n * n * bi;
    rep->launches += 2;

  }
  return MBINV_OK;
}

static mbinv_status mbinv_backward_impl(mbinv_ctx* c, int64_t i, int64_t j, const void* G, int64_t ldg, void* dM,
                                        int64_t ldd, mbinv_report* rep) {
  if (!c || !G || !dM || i < 0 || j < 0 || i >= c->k || j >= c->k || ldd < c->n) return MBINV_EINVAL;
  if (ldg < block_extent(c, j)) return MBINV_EINVAL;
  start_report(rep);
  // the FP64-valued paths: rows, columns and products in FP64 (digit products
  // on FP64_TC), optionally refined; the FP32-valued paths in M's type
  if (c->opt.precision == MBINV_FP64 || c->opt.precision == MBINV_FP64_TC)
    return backward_fp64(c, i, j, G, ldg, dM, ldd, rep);
  return backward_same_type(c, i, j, G, ldg, dM, ldd, rep);
}

static mbinv_status mbinv_batched_blocks_impl(int64_t count, mbinv_problem* probs, int dtype, const mbinv_options* opt,
                                  mbinv_report* rep) {
  if (count < 0 || (count > 0 && !probs)) return MBINV_EINVAL;
  if (dtype != F64 && dtype != F32) return MBINV_EINVAL;
  start_report(rep);
  if (count == 0) return MBINV_OK;
  auto t0 = std::chrono::steady_clock::now();
  mbinv_options o;
  mbinv_default_options(&o);
  if (opt) {
    if (opt->struct_size != sizeof(mbinv_options)) return MBINV_EINVAL;
    o = *opt;
  }
  if (o.refine_steps > 0) return MBINV_ENOTSUP;
  // one context per problem (its device matrix and plan), all run together;
  // their device bytes and the shared executor's are counted together
  MemTrack shared;
  std::vector<mbinv_ctx*> ctxs((size_t)count, nullptr);
  mbinv_status first = MBINV_OK;
  auto cleanup = [&]() {
    for (mbinv_ctx* c : ctxs) mbinv_destroy(c);
  };
  for (int64_t t = 0; t < count; ++t) {
    mbinv_problem& p = probs[t];
    p.status = MBINV_EINVAL;
    if (p.i < 0 || p.j < 0 || p.i >= p.k || p.j >= p.k || !p.out) continue;
    p.status = guarded([&] { return mbinv_create_impl(&ctxs[t], p.n, p.k, dtype, p.M, p.ld, &o, &shared); });
  }
  // run in waves whose summed workspace fits the cap
  Env env;
  for (DevBuf* d : env.bufs()) d->track = &shared;
  env.stream = (cudaStream_t)o.cuda_stream;
  env.precision = o.precision;
  env.slices = o.bf16_slices;
  env.profile = o.profile != 0;
  env.sing_tol = o.sing_tol;
  env.pivot_cond = o.pivot_cond != 0;
  env.use_graphs = false;  // every wave is a different launch sequence
  std::vector<int64_t> order;
  for (int64_t t = 0; t < count; ++t)
    if (ctxs[t] && probs[t].status == MBINV_OK) order.push_back(t);
  size_t q0 = 0, peak = 0;
  while (q0 < order.size()) {
    std::vector<Job> jobs;
    std::vector<int64_t> members;
    size_t used = 0;
    int ic = INT_MAX;
    int64_t bmax_wave = 1;
    size_t q = q0;
    for (; q < order.size(); ++q) {
      mbinv_ctx* c = ctxs[order[q]];
      mbinv_problem& p = probs[order[q]];
      const Schedule* S;
      if (get_plan(c, {{(int)p.i, (int)p.j}}, &S) != MBINV_OK) {
        p.status = MBINV_ENOMEM_CAP;
        continue;
      }
      const size_t need = run_bytes(c, *S, S->inv_chunk) + c->own_M.bytes;
      if (!jobs.empty() && ((o.device_cap_bytes && used + need > o.device_cap_bytes) || jobs.size() >= 1024)) break;
      if (set_border(c, border_of(c, p.i, p.j)) != MBINV_OK ||
          c->slots.ensure((size_t)S->nslots * slot_bytes_for((int)c->b, o.precision)) != cudaSuccess ||
          c->outtmp.ensure((size_t)c->b * c->b * 8 + 256) != cudaSuccess) {
        p.status = MBINV_ECUDA;
        continue;
      }
      used += need;
      // without a cap every member's inverses of a step share one launch
      // sequence; under a cap each member keeps the chunk that fits it
      ic = o.device_cap_bytes ? std::min(ic, S->inv_chunk) : (ic == INT_MAX ? 0 : ic) + S->inv_chunk;
      bmax_wave = std::max<int64_t>(bmax_wave, c->b);
      Job J;
      J.dM = c->dM;
      J.ldm = c->ldm;
      J.mdt = c->mdt;
      J.b = (int)c->b;
      J.slots = (char*)c->slots.p;
      J.slot_bytes = slot_bytes_for((int)c->b, o.precision);
      J.slot_dt = env_slot_type(o.precision);
      J.out = c->outtmp.p;
      J.ldo = c->b;
      J.out_dt = dtype;
      J.S = S;
      jobs.push_back(J);
      members.push_back(order[q]);
      if (rep) add_report(rep, c, *S);
    }
    q0 = q;
    if (members.empty()) continue;
    env.inv_chunk = std::max(1, std::min(ic, max_inv_chunk((int)bmax_wave, o.precision)));
    mbinv_status s = run_jobs(env, jobs);
    if (s == MBINV_ECUDA) {
      last_cuda_error() = env.last_error;
      for (int64_t t : members) probs[t].status = MBINV_ECUDA;
    } else {
      for (size_t u = 0; u < members.size(); ++u) {
        mbinv_problem& p = probs[members[u]];
        mbinv_ctx* c = ctxs[members[u]];
        if (env.job_singular[u]) {
          p.status = MBINV_ESINGULAR;
          continue;
        }
        if (s == MBINV_ETIMEOUT) {
          p.status = MBINV_ETIMEOUT;
          continue;
        }
        const int64_t bi = block_extent(c, p.i), bj = block_extent(c, p.j);
        const size_t es = dtype_size(dtype);
        const bool dev = is_device_ptr(p.out);
        p.status = cudaMemcpy2DAsync(p.out, (size_t)p.ldo * es, c->outtmp.p, (size_t)c->b * es, (size_t)bj * es,
                                     (size_t)bi, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                     env.stream) == cudaSuccess
                       ? MBINV_OK
                       : MBINV_ECUDA;
      }
      cudaStreamSynchronize(env.stream);
    }
    if (rep) {
      rep->launches += env.launches;
      rep->gemm_launches += env.gemm_launches;
      rep->max_pivot_cond = std::max(rep->max_pivot_cond, env.max_cond);
      add_env_report(rep, env);
    }
    peak = std::max(peak, used);
    // the finished members' device memory goes before the next wave
    for (int64_t t : members) {
      mbinv_destroy(ctxs[t]);
      ctxs[t] = nullptr;
    }
  }
  env.release();
  cleanup();
  for (int64_t t = 0; t < count; ++t)
    if (probs[t].status != MBINV_OK && first == MBINV_OK) first = (mbinv_status)probs[t].status;
  if (rep) {
    rep->peak_device_bytes = shared.hwm;
    rep->planned_device_bytes = peak;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return first;
}

static mbinv_status mbinv_autotune_impl(int64_t b, int64_t count, int precision, const char* path, int* best_bias,
                                        double* best_seconds) {
  if (b < 1 || count < 1 || count > (1 << 20) || precision < MBINV_FP64 || precision > MBINV_FP64_TC ||
      precision == MBINV_MIXED_BF16)
    return MBINV_EINVAL;
  const int wt = env_work_type(precision);
  const bool tc = precision == MBINV_FP64_TC;
  DevBuf A, O;
  const size_t bytes = (size_t)count * b * b * 8;
  CU(A.ensure(bytes));
  CU(O.ensure(bytes));
  tune_fill_kernel<<<(unsigned)((count * b * b + 255) / 256), 256>>>((double*)A.p, count, b);
  CU(cudaGetLastError());
  CU(cudaDeviceSynchronize());
  std::vector<mbinv_problem> probs((size_t)count);
  for (int64_t t = 0; t < count; ++t)
    probs[t] = mbinv_problem{b, 1, 0, 0, (double*)A.p + t * b * b, b, (double*)O.p + t * b * b, b, 0};
  mbinv_options o;
  mbinv_default_options(&o);
  o.precision = (mbinv_precision)precision;
  o.profile = 1;
  int best = 0;
  double best_t = 1e300;
  for (int bias : {0, -1, 1, -2, 2}) {
    set_cluster_bias((int)b, (int)count, wt, tc, bias);
    double t = 0;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
      mbinv_report r;
      const mbinv_status s = mbinv_batched_blocks(count, probs.data(), F64, &o, &r);
      if (s != MBINV_OK) {
        set_cluster_bias((int)b, (int)count, wt, tc, 0);
        return s;
      }
      t = r.inv_device_seconds;
    }
    if (t < best_t) {
      best_t = t;
      best = bias;
    }
  }
  set_cluster_bias((int)b, (int)count, wt, tc, best);
  if (path) {
    FILE* f = fopen(path, "a");
    if (!f) return MBINV_EINVAL;
    fprintf(f, "%lld %lld %d %d %.9g\n", (long long)b, (long long)count, precision, best, best_t);
    fclose(f);
  }
  if (best_bias) *best_bias = best;
  if (best_seconds) *best_seconds = best_t;
  return MBINV_OK;
}

mbinv_status mbinv_autotune(int64_t b, int64_t count, int precision, const char* path, int* best_bias,
                            double* best_seconds) {
  return guarded([&] { return mbinv_autotune_impl(b, count, precision, path, best_bias, best_seconds); });
}

mbinv_status mbinv_create(mbinv_ctx** out, int64_t n, int64_t k, int dtype, const void* M, int64_t ld,
                          const mbinv_options* opt) {
  return guarded([&] { return mbinv_create_impl(out, n, k, dtype, M, ld, opt); });
}
mbinv_status mbinv_create_from_fn(mbinv_ctx** out, int64_t n, int64_t k, int dtype, mbinv_block_fn fn, void* user,
                                  const mbinv_options* opt) {
  return guarded([&] { return mbinv_create_from_fn_impl(out, n, k, dtype, fn, user, opt); });
}
mbinv_status mbinv_reload(mbinv_ctx* c) {
  return on_context(c, nullptr, [&]() -> mbinv_status {
    // a context that copied M re-reads it; one that reads the caller's
    // buffer in place (device M, host-resident M) or produces M has nothing
    // to refresh
    if (!c->own_M.p || !c->srcM) return MBINV_OK;
    return upload_m(c, c->own_M.track);
  });
}
mbinv_status mbinv_block(mbinv_ctx* c, int64_t i, int64_t j, void* out, int64_t ldo, mbinv_report* rep) {
  return on_context(c, rep, [&] { return mbinv_block_impl(c, i, j, out, ldo, rep); });
}
mbinv_status mbinv_blocks(mbinv_ctx* c, int64_t count, const int64_t* ij, void* const* outs, const int64_t* ldos,
                          int width, mbinv_report* rep) {
  return on_context(c, rep, [&] { return mbinv_blocks_impl(c, count, ij, outs, ldos, width, rep); });
}
mbinv_status mbinv_all_blocks(mbinv_ctx* c, void* out, int64_t ldo, const uint8_t* done, mbinv_block_done_cb cb,
                              void* user, mbinv_report* rep) {
  return on_context(c, rep, [&] { return mbinv_all_blocks_impl(c, out, ldo, done, cb, user, rep); });
}
mbinv_status mbinv_block_row(mbinv_ctx* c, int64_t i, void* out, int64_t ldo, mbinv_report* rep) {
  return on_context(c, rep, [&] { return mbinv_block_row_impl(c, i, out, ldo, rep); });
}
mbinv_status mbinv_block_col(mbinv_ctx* c, int64_t j, void* out, int64_t ldo, mbinv_report* rep) {
  return on_context(c, rep, [&] { return mbinv_block_col_impl(c, j, out, ldo, rep); });
}
mbinv_status mbinv_backward(mbinv_ctx* c, int64_t i, int64_t j, const void* G, int64_t ldg, void* dM, int64_t ldd,
                            mbinv_report* rep) {
  return on_context(c, rep, [&] { return mbinv_backward_impl(c, i, j, G, ldg, dM, ldd, rep); });
}
mbinv_status mbinv_batched_blocks(int64_t count, mbinv_problem* probs, int dtype, const mbinv_options* opt,
                                  mbinv_report* rep) {
  return guarded([&] { return mbinv_batched_blocks_impl(count, probs, dtype, opt, rep); });
}

}  // extern "C"
