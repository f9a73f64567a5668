// Executor of recursion schedules: one or many independent requests run
// together, level by level, in grouped launches on one stream.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <vector>

#include "../../include/mbinv.h"
#include "mbinv_internal.h"

namespace mbinv {

// Device bytes a context holds, counted at every allocation and free, and
// the bound they must stay under (0 = none).
struct MemTrack {
  size_t live = 0, hwm = 0, cap = 0;
};

// Set when an allocation was refused because it would have crossed the cap
// (the caller then reports MBINV_ENOMEM_CAP rather than a CUDA error).
inline bool& cap_refused() {
  static thread_local bool f = false;
  return f;
}

// Test hook: the next n device allocations of the library fail as if the
// device were out of memory (cudaErrorMemoryAllocation), before cudaMalloc.
// One counter per process (defined once, in exec.cu).
std::atomic<int>& injected_alloc_failures();

// A device buffer that grows on demand.  With a tracker attached, every byte
// it holds is counted there, and growth that would take the tracker past its
// cap is refused before cudaMalloc is called.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  MemTrack* track = nullptr;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    release();
    if (track && track->cap && track->live + need > track->cap) {
      cap_refused() = true;
      return cudaErrorMemoryAllocation;
    }
    if (injected_alloc_failures().load() > 0 && injected_alloc_failures().fetch_sub(1) > 0)
      return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = need;
    if (track) {
      track->live += need;
      track->hwm = track->live > track->hwm ? track->live : track->hwm;
    }
    return cudaSuccess;
  }
  void release() {
    if (p) {
      cudaFree(p);
      if (track) track->live -= bytes;
    }
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

// One job: the matrix it reads, its value slots, its outputs (one per request
// of its plan), its schedule.
struct Job {
  const void* dM = nullptr;  // (bordered) matrix, row-major
  int64_t ldm = 0;
  int mdt = F64;
  int b = 0;
  char* slots = nullptr;     // this request's slots, slot_bytes apart
  size_t slot_bytes = 0;
  int slot_dt = F64;
  void* out = nullptr;       // device destination of N_ij (b x b), one request
  int64_t ldo = 0;
  std::vector<void*> outs;   // several requests: destination of request r
  std::vector<int64_t> ldos;
  // bounded schedules: the matrix in host memory (HOSTM copies) and the host
  // spill area (SPILL slots, slot_bytes apart)
  const void* hM = nullptr;
  int64_t hldm = 0;
  int hmdt = F64;
  char* spill = nullptr;
  // a produced matrix: HOSTM blocks are written by gen instead of copied
  mbinv_block_fn gen = nullptr;
  void* gen_user = nullptr;
  int out_dt = F64;
  const Schedule* S = nullptr;
};

// Buffers and settings shared by the requests of one run.
struct Env {
  cudaStream_t stream = nullptr;
  int precision = MBINV_FP64;
  int slices = 3;
  bool profile = false;
  int inv_chunk = 1;  // matrices per inverse launch
  DevBuf inv_work, inv_wrow, inv_perm, inv_amax, inv_tc, desc, status, flags, apk, bpk, b2pk, tcerr, oexp;
  DevBuf stage;        // a block of a host matrix on its way to a slot of another type
  DevBuf condw;        // largest condition estimate of the run's inverses (bits of a double)
  double sing_tol = 0; // relative singularity threshold of the pivots (0 = b eps)
  bool pivot_cond = false;  // estimate every inverted pivot's condition
  // CUDA graph of the last repeated launch sequence (see run_jobs)
  bool use_graphs = true;
  cudaStream_t cstream = nullptr;  // capture stream
  cudaGraphExec_t gexec = nullptr;
  std::vector<uintptr_t> gkey;
  std::vector<char> garena;
  int glaunches = 0, ggemm_launches = 0;
  size_t gpused = 0;
  size_t graph_replays = 0;
  double max_cond = 0; // of the last run
  HostBuf hdesc;
  std::vector<cudaEvent_t> events;
  // results of the last run
  int launches = 0, gemm_launches = 0;
  double host_in_bytes = 0, host_out_bytes = 0;  // copies of the last run
  double gemm_dev_s = 0, inv_dev_s = 0, pack_dev_s = 0;
  double pack_bytes = 0;  // algorithmic bytes of the operand packs of the last run
  double inv_panel_dev_s = 0, inv_panel_flops = 0, inv_update_flops = 0;
  size_t inv_panel_launches = 0;
  std::vector<cudaEvent_t> pevents;  // panel timing (profile)
  // buffers of the sweep (everything but the descriptor staging on the host)
  std::vector<DevBuf*> bufs() {
    return {&inv_work, &inv_wrow, &inv_perm, &inv_amax, &inv_tc, &desc,  &status, &flags,
            &apk,      &bpk,      &b2pk,     &tcerr,    &oexp,   &stage, &condw};
  }
  std::vector<int> job_singular;  // per job
  int64_t failed_inverse = -1;    // first singular inverse, in launch order
  cudaError_t last_error = cudaSuccess;

  void release();
};

inline int env_work_type(int precision) { return precision == MBINV_FP32 ? F32 : F64; }
inline int env_slot_type(int precision) {
  return (precision == MBINV_FP64 || precision == MBINV_FP64_TC) ? F64 : F32;
}
size_t slot_bytes_for(int b, int precision);
// Device bytes of inverse scratch for count matrices of order at most bmax.
size_t inv_scratch_bytes(int bmax, int precision, int count);
// Device bytes of the packed operand slabs of the mixed path for a run whose
// widest GEMM step has `ops` products of order bmax.
size_t pack_bytes(int bmax, int slices, size_t ops);
// Device bytes of the digit slabs and row exponents of the FP64_TC path for a
// run whose widest GEMM step has `ops` products of order bmax.
size_t digit_bytes(int bmax, size_t ops);
// Device bytes of the executor's descriptor arena, operand slabs and staging
// for one job running schedule S at order b (what run_jobs allocates beside
// the value slots and the inverse scratch).
size_t arena_bytes(const Schedule& S, int b, int precision, int slices, int inv_chunk, int host_dt, int slot_dt);

// Runs the schedules of `jobs` together: step t of every schedule goes out in
// the same grouped launches.  Returns MBINV_ESINGULAR if any request met a
// singular pivot (E.job_singular says which).
mbinv_status run_jobs(Env& E, const std::vector<Job>& jobs);

}  // namespace mbinv
