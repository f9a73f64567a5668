// Internal declarations shared by the translation units of libmbinv.
// Nothing here is part of the public C ABI (include/mbinv.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

namespace mbinv {

enum DType : int { F64 = 0, F32 = 1, BF16 = 2 };

inline size_t dtype_size(int t) { return t == F64 ? 8 : (t == F32 ? 4 : 2); }

// Runs setup once per (key, current device) - a kernel's shared-memory
// attribute, say - safely for several host threads and several devices;
// retried on a later call if it failed.
cudaError_t once_per_device(const void* key, const std::function<cudaError_t()>& setup);
// Multiprocessors of the current device.
int sm_count();

// --------------------------------------------------------------- planner
// A frame of the recursion (Sec. 3.1) after hash-consing: its value is
//   order 2 (leaf):  M[krow, kcol] - M[krow, pcol] (P^-1 M[prow, kcol]),
//                    P = M[prow, pcol] the pivot block of the request that
//                    reached it (Eqs. FA2-FD2);
//   order >= 3:      kept - left * (piv^-1 * right), the four operands being
//                    frames of the order below, chosen by the frame's role
//                    (Eqs. SchurofA-SchurofD).
// Two frames are one when they compute the same thing: leaves with the same
// (krow, kcol, prow, pcol), other frames with the same four operand frames.
// Such frames round identically, so sharing them across requests changes no
// bit of any result.
struct PFrame {
  int order = 0;
  int krow = -1, kcol = -1, prow = -1, pcol = -1;  // leaves
  int kept = -1, left = -1, piv = -1, right = -1;  // order >= 3
};

struct Plan {
  int k = 0;
  std::vector<std::pair<int, int>> reqs;  // requested blocks (i, j), 0-based
  std::vector<int> roots;                 // frame id of each request's root
  std::vector<PFrame> f;
  std::vector<std::vector<int>> level;    // level[p] = ids of frames of order p
  size_t nonleaf = 0, leaves = 0;
  size_t request_frames = 0;              // sum over requests of their own distinct frames
};

// The frame DAG of several requests on one k x k grid, built request by
// request as the paper's forward procedure prescribes and merged by value.
Plan build_plan(int k, const std::vector<std::pair<int, int>>& reqs, bool pad_last);
inline Plan build_plan(int k, int i, int j, bool pad_last) { return build_plan(k, {{i, j}}, pad_last); }

// Operand reference of a scheduled operation.
struct Ref {
  // MBLK: block (r, c) of the device matrix; SLOT: a device value slot; OUT:
  // a request's output; HOSTM: block (r, c) of the matrix kept in host
  // memory; SPILL: a slot of the host spill area
  enum Kind : int { NONE = 0, MBLK = 1, SLOT = 2, OUT = 3, HOSTM = 4, SPILL = 5 } kind = NONE;
  int r = 0, c = 0;  // block coordinates for MBLK / HOSTM
  int slot = -1;     // slot id for SLOT / SPILL; request index for OUT
};

struct GemmOp {  // C = alpha * A * B + beta * Cin, all b x b
  Ref A, B, Cin, C;
  double alpha = 1.0, beta = 0.0;
};
struct InvOp {  // dst = src^-1
  Ref src, dst;
  int frame = -1;
};
struct CopyOp {  // dst = src (host <-> device), b x b
  Ref src, dst;
};
struct Step {
  // COPY: values moved between host memory and device slots (a block of a
  // host-resident M loaded, a value spilled to the host or brought back)
  enum Kind : int { INV = 0, GEMM = 1, COPY = 2 } kind = INV;
  std::vector<InvOp> inv;
  std::vector<GemmOp> gemm;
  std::vector<CopyOp> copy;
};

struct Schedule {
  std::vector<Step> steps;
  int nouts = 1;       // requests: Ref::OUT's slot field indexes them
  int nslots = 0;      // peak number of b x b value slots alive at once
  int max_inv_batch = 0;
  double gemm_flops_units = 0;  // in units of b^3 (2 per product)
  double inv_units = 0;         // in units of b^3 (2 per inverse)
  size_t frames = 0, inversions = 0;
  size_t request_frames = 0;    // frames the requests would evaluate one by one
  int inv_chunk = 0;            // matrices per inverse launch chosen to fit the cap
  size_t planned = 0;           // device bytes of its workspace with that chunk
  // bounded schedules (build_bounded_schedule)
  bool bounded = false;
  int nspill = 0;               // host spill slots needed at once
  size_t loads = 0, spills = 0; // b x b copies host -> device and device -> host
};

// Builds the level-by-level schedule of a plan (one or several requests).
// zchunk bounds the number of Schur temporaries alive at once (0 = a whole
// level).
Schedule build_schedule(const Plan& p, int zchunk);

// The memory-bounded schedule of a plan: frames evaluated depth first, one
// operation per step, in at most `slots` device value slots.  The blocks of M
// come from host memory when host_m (HOSTM copies) and from the device
// matrix otherwise; a value evicted while it is still needed is spilled to
// a host slot and copied back before its next use, the victim being the value
// needed again last (Belady's rule on the known sequence).  Returns false
// when `slots` is too small for a single operation.
bool build_bounded_schedule(const Plan& p, int slots, bool host_m, Schedule* out);

// The principal-Schur-complement variant of block (i, j) (see plan.cpp): the
// other blocks eliminated in ascending order with principal pivots, then the
// 2 x 2 (or 1 x 1) remainder inverted.  One request; its output is OUT 0.
Schedule build_psc_schedule(int k, int i, int j);

// --------------------------------------------------------------- kernels
struct GemmDesc {
  const void* A;
  const void* B;
  const void* Cin;
  void* C;
  int64_t lda, ldb, ldcin, ldc;
  int m, n, k;
  int ta, tb;      // op(A) = A^T when ta, op(B) = B^T when tb
  double alpha, beta;
  int tiles_n;     // column tiles of this problem
  int tile_start;  // first global tile index of this problem
};

// Element-type combination of a grouped GEMM: A, B, C types and the
// accumulator's.
enum GemmCombo : int {
  G_F64 = 0,       // double x double -> double, FP64 accumulate
  G_F32 = 1,       // float x float -> float, FP32 accumulate
  G_F32IN_F64 = 2, // float x float -> double, FP64 accumulate
  G_F64F32_F64 = 3, // double x float -> double, FP64 accumulate
  G_F32F64_F64 = 4  // float x double -> double, FP64 accumulate
};
void gemm_tile_shape(int combo, int* bm, int* bn);
cudaError_t launch_gemm_grouped(int combo, const GemmDesc* d_descs, int ndesc, int total_tiles, cudaStream_t s);

// Batched Gauss-Jordan inversion with partial pivoting.
struct InvDesc {
  const void* src;  // input matrix (b x b, leading dimension lds)
  int64_t lds;
  void* dst;        // output (b x b, leading dimension ldd)
  int64_t ldd;
  void* work;       // b x b scratch in the working precision
  void* wrow;       // nb x b scratch: pivot rows of the trailing columns
  int* perm;        // b ints: row interchanges
  unsigned long long* amax;  // max |entry| (bit pattern of a non-negative double)
  int b;
  int tag;          // reported through the status word when singular
  int* flag;        // set to 1 when singular (may be null): per-problem status
  double tol_rel;   // a pivot is singular at or below tol_rel * max|entry|;
                    // 0 = b times the unit roundoff of the working type
  unsigned long long* cond;  // if set: max with the bits of ||src||_1 ||dst||_1
};

// Largest 1-norm condition estimate ||src||_1 ||dst||_1 of count inverted
// matrices, folded (as the bit pattern of a non-negative double) into each
// descriptor's cond word.
cudaError_t launch_cond1(const InvDesc* d_desc, int count, int in_dtype, int out_dtype, cudaStream_t s);
// Status word written by the inverse kernels: flag != 0 when a pivot was
// singular; tag holds the smallest failing InvDesc::tag.
struct DevStatus {
  int singular;
  int tag;
};
// Panel width of the blocked elimination for order b in working type wtype
// (tc: the trailing update runs on the tensor cores, which favour 64).
int inv_panel_width(int b, int wtype, bool tc = false);
// Device scratch of the tensor-core trailing update for count FP64 matrices
// of order at most bmax: digit slabs of the panel columns and of the pivot
// rows, their exponents, and the per-matrix descriptors.
struct InvTc {
  void* scratch;  // inv_tc_bytes(bmax, count) bytes, 256-byte aligned
  int* err;       // raised when a wait of the product kernel ran out
};
size_t inv_tc_bytes(int bmax, int count);
// Optional timing of run_inverse_batch: an event is recorded before and after
// every panel launch (ev[n], ev[n + 1], n += 2) while n + 2 <= cap.
struct InvTiming {
  cudaEvent_t* ev;
  int cap;
  int n;
};
// Tuned panel-cluster bias for inverse batches of count matrices of order b
// (the cluster the heuristic picks is scaled by 2^bias, within the shared-
// memory limit); 0 until set.  Thread safe.
void set_cluster_bias(int b, int count, int wtype, bool tc, int bias);
int cluster_bias(int b, int count, int wtype, bool tc);
// Panel width and algorithmic flops of the panel factorisations and of the
// trailing updates of one inverse of order b.
void inv_flop_split(int b, int wtype, bool tc, double* panel_flops, double* update_flops);
// Inverts count matrices described by d_desc; b is the largest order among
// them (each descriptor carries its own).  in_dtype / out_dtype / wtype are
// DType values; wtype is F64 or F32.  The max|entry| words are zeroed by the
// call.  With tc (FP64 only) the trailing updates are exact digit products
// on the tensor cores instead of FP64 tile products.
cudaError_t run_inverse_batch(int in_dtype, int out_dtype, int wtype, const InvDesc* d_desc, int count, int b,
                              DevStatus* d_status, cudaStream_t s, int* launches, const InvTc* tc = nullptr,
                              InvTiming* timing = nullptr);

}  // namespace mbinv
