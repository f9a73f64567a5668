// Batched b x b inverse by Gauss-Jordan elimination with partial pivoting.
//
// The paper inverts each b x b pivot with an LU routine that pivots by row
// interchanges (Sec. 5 and Sec. 7).  Gauss-Jordan with partial pivoting picks
// the same pivots as LU with partial pivoting (the candidates of column j are
// the entries of the current Schur complement) and produces the inverse in
// place; its 2 b^3 flops are the paper's "O(b^3)" per inversion (Sec. 6,
// property (b)).
//
// Blocked in-place form, panel width nb.  For the panel J = [p, p + nb):
//   1. panel kernel (one CTA per matrix): for each column j of J, pick the
//      first row r >= j of largest |x_rj|, exchange whole rows j and r,
//      scale row j and eliminate column j from every other row - on the
//      panel columns only.  The panel then holds T[:, J], where T is the
//      product of the nb elementary transforms; the pivot rows of the other
//      columns are copied to a scratch W = X[J, rest].
//   2. update kernel (many CTAs per matrix): X[:, rest] = T[:, J] W + X[:, rest]
//      with the rows of J zeroed first - a rank-nb GEMM on the CUDA cores,
//      or (FP64_TC) an exact digit product on the tensor cores (ozaki.cu):
//      T[:, J] by rows and W by columns are digit-packed and one grouped
//      product forms the update in FP64.  On FP64_TC the update is delayed
//      over blocks of two panels (K = 2 nb; each panel's columns are brought
//      up to date with the earlier panels of its block before it, and the
//      earlier panels' columns take its transform after it - narrow
//      products), see run_batch_t.
// After the last panel the recorded row interchanges are undone as column
// interchanges in reverse order while the result is written out.  For b at
// most 128 the panel is the whole matrix and step 2 never runs.
//
// A pivot whose magnitude is not finite or is <= b * eps * max|entry| marks
// the matrix singular through the status word; the elimination still runs to
// the end so that no thread waits on another.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cfloat>

#include "mbinv_internal.h"
#include "ozaki.h"
#include "tile_gemm.cuh"

#include <cooperative_groups.h>

namespace mbinv {

namespace {

constexpr int kPanelThreads = 256;
constexpr int kMaxPanelWidth = 256;
constexpr int kSmemLimit = 200 * 1024;

template <typename TW>
__device__ __forceinline__ TW eps_of();
template <>
__device__ __forceinline__ double eps_of<double>() { return DBL_EPSILON; }
template <>
__device__ __forceinline__ float eps_of<float>() { return FLT_EPSILON; }

__global__ void zero_amax_kernel(const InvDesc* __restrict__ d, int count) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) *d[t].amax = 0ull;
}

// work = (TW) src; amax = max |src| as the bit pattern of a non-negative
// double: the integer order of those patterns is their numeric order, and a
// NaN's pattern is above every number's, which makes the matrix singular.
// CTA x takes rows x, x + gridDim.x, ..., its threads the columns; the
// maximum is kept on the bit patterns (integer instructions, no FP64).
template <typename TW, typename TI>
__device__ __forceinline__ unsigned long long init_rows(const InvDesc& d, const TI* __restrict__ src, TW* w) {
  const int b = d.b;
  unsigned long long m = 0;
  for (int r = blockIdx.x; r < b; r += gridDim.x) {
    const TI* s = src + (int64_t)r * d.lds;
    TW* o = w + (int64_t)r * b;
    for (int c = threadIdx.x; c < b; c += blockDim.x) {
      const double v = (double)s[c];
      o[c] = (TW)v;
      const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
      m = a > m ? a : m;
    }
  }
  return m;
}

template <typename TW>
__global__ void gj_init_kernel(const InvDesc* __restrict__ descs, int in_dtype) {
  const InvDesc d = descs[blockIdx.y];
  TW* w = (TW*)d.work;
  unsigned long long m = in_dtype == F64 ? init_rows<TW>(d, (const double*)d.src, w)
                                         : init_rows<TW>(d, (const float*)d.src, w);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, m, o);
    m = x > m ? x : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(d.amax, m);
}

// Pivot keys: the bit pattern of |x| orders like |x| for every non-NaN x, and
// a NaN maps to -1 so that it never wins; comparing keys keeps the pivot
// search off the FP64 pipe (which takes a whole warp instruction even for
// one active lane).
__device__ __forceinline__ long long pivot_key(double v) {
  const long long a = __double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFLL;
  return a > 0x7FF0000000000000LL ? -1LL : a;
}
__device__ __forceinline__ long long pivot_key(float v) {
  const int a = __float_as_int(v) & 0x7FFFFFFF;
  return a > 0x7F800000 ? -1LL : (long long)a;
}
__device__ __forceinline__ double key_value(long long k, double) {
  return k < 0 ? __longlong_as_double(0x7FF8000000000000LL) : __longlong_as_double(k);
}
__device__ __forceinline__ float key_value(long long k, float) {
  return k < 0 ? __int_as_float(0x7FC00000) : __int_as_float((int)k);
}

// Warp-wide argmax of (key, row): the largest key, and among equal keys the
// smallest row, in three warp reductions (the key's high word, its low word
// among the lanes that hold the largest high word, then the row).
__device__ __forceinline__ void warp_argmax(long long& key, int& row) {
  const int hi = (int)(key >> 32);
  const unsigned lo = (unsigned)key;
  const int mh = __reduce_max_sync(0xffffffffu, hi);
  const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
  row = __reduce_min_sync(0xffffffffu, (hi == mh && lo == ml) ? row : 0x7fffffff);
  key = (long long)(((unsigned long long)(unsigned)mh << 32) | ml);
}

// A cluster of CL CTAs per matrix factors the panel [p, p + nb) (see the file
// comment).  CTA q of the cluster keeps rows [row0 + q R, row0 + (q+1) R) of
// the panel in its shared memory (R = ceil((b - row0) / CL)); the CTAs
// exchange pivot candidates and the pivot row through distributed shared
// memory, so that the per-column work (the elimination of nb columns from
// every row) is spread over CL SMs instead of one.  Every warp of every CTA
// takes the same pivot decision from the same candidates, so one column costs
// two CTA barriers and two cluster barriers (CTA barriers when CL = 1).
template <typename TW>
__global__ void __launch_bounds__(kPanelThreads) gj_panel_kernel(const InvDesc* __restrict__ descs, int p, int nb,
                                                                 DevStatus* status, int active_only) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NW = kPanelThreads / 32;
  const int CL = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  const InvDesc d = descs[blockIdx.x / CL];
  const int b = d.b;
  // a cluster of one CTA synchronises as a CTA
  auto csync = [&]() {
    if (CL == 1)
      __syncthreads();
    else
      cluster.sync();
  };
  // matrices of a batch may differ in order: this one's panel may be narrower
  // or already past its end (the whole cluster leaves together)
  const int ldp = nb + 1;  // odd stride: a column read by consecutive rows spreads over banks
  nb = min(nb, b - p);
  if (nb <= 0) return;
  // rows the panel eliminates: all of them, or (active_only) only the rows
  // not yet used as pivots, [p, b) - the others' panel columns then follow
  // from one product with the inverse of the pivot block (see run_batch_t)
  const int row0 = active_only ? p : 0;
  const int R = (b - row0 + CL - 1) / CL;
  const int r0 = min(b, row0 + q * R), r1 = min(b, r0 + R);
  TW* P = (TW*)smem_raw;                // P[(i - r0) * ldp + t] is X[i][p + t]
  TW* prow = P + (size_t)R * ldp;       // pivot row before scaling (nb)
  TW* jrow = prow + ldp;                // old row j, for the owner of row r (nb)
  TW* srow = jrow + ldp;                // scaled pivot row (nb)
  int* piv_hist = (int*)(srow + ldp);   // pivot row of every column of the panel (nb)
  __shared__ long long cand_v[2][NW];
  __shared__ int cand_i[2][NW];
  TW* X = (TW*)d.work;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < (r1 - r0) * nb; e += kPanelThreads) {
    const int i = e / nb, t = e % nb;
    P[i * ldp + t] = X[(int64_t)(r0 + i) * b + p + t];
  }
  const double amax = __longlong_as_double((long long)*d.amax);
  const TW tol = (TW)((d.tol_rel > 0.0 ? d.tol_rel : (double)b * (double)eps_of<TW>()) * amax);
  __syncthreads();

  for (int t = 0; t < nb; ++t) {
    const int j = p + t;
    const int buf = t & 1;
    // ---- this warp's pivot candidate: first row of largest magnitude, rows >= j
    {
      long long best = -1;
      int bi = b;
      for (int i = max(j, r0) + tid; i < r1; i += kPanelThreads) {
        const long long v = pivot_key(P[(i - r0) * ldp + t]);
        if (v > best) { best = v; bi = i; }  // NaN never wins
      }
      warp_argmax(best, bi);
      if (lane == 0) { cand_v[buf][warp] = best; cand_i[buf][warp] = bi; }
    }
    csync();  // #1: the candidates of every warp of every CTA are visible
    // ---- global pivot, computed by every warp from the same CL x NW candidates
    int r;
    long long gk;
    {
      long long v = -1;
      int ix = b;
      for (int u = lane; u < CL * NW; u += 32) {
        const long long cv = *cluster.map_shared_rank(&cand_v[buf][u % NW], u / NW);
        const int ci = *cluster.map_shared_rank(&cand_i[buf][u % NW], u / NW);
        if (cv > v || (cv == v && ci < ix)) { v = cv; ix = ci; }
      }
      warp_argmax(v, ix);
      r = ix >= b ? j : ix;  // every candidate NaN: keep the row
      gk = v;
    }
    if (tid == 0) {
      piv_hist[t] = r;
      if (q == 0) {
        const TW gv = key_value(gk, (TW)0);
        if (!(gv > tol) || !isfinite((double)gv)) {
          atomicExch(&status->singular, 1);
          atomicMin(&status->tag, d.tag);
          if (d.flag) atomicExch(d.flag, 1);
        }
        d.perm[j] = r;
      }
    }
    const int oj = (j - row0) / R, orr = (r - row0) / R;  // owners of rows j and r
    // ---- read the pivot row (old row r) and, for the owner of r, old row j
    {
      const TW* src = cluster.map_shared_rank(P, orr) + (size_t)(r - row0 - orr * R) * ldp;
      for (int c = tid; c < nb; c += kPanelThreads) prow[c] = src[c];
      if (q == orr && r != j) {
        const TW* sj = cluster.map_shared_rank(P, oj) + (size_t)(j - row0 - oj * R) * ldp;
        for (int c = tid; c < nb; c += kPanelThreads) jrow[c] = sj[c];
      }
    }
    csync();  // #2: every CTA has read rows j and r; prow and jrow are complete
    // ---- scale the pivot row and eliminate column j (warp per row, lane per
    // column).  Row j receives the scaled pivot row; row r, when it moved,
    // starts from the old row j (jrow).
    // the scaled pivot row, once per CTA (FP64 divisions are dear: one per column)
    const TW piv = prow[t];
    for (int c = tid; c < nb; c += kPanelThreads) srow[c] = ((c == t) ? (TW)1 : prow[c]) / piv;
    __syncthreads();
    for (int i = r0 + warp; i < r1; i += NW) {
      TW* xi = P + (size_t)(i - r0) * ldp;
      if (i == j) {
        for (int c = lane; c < nb; c += 32) xi[c] = srow[c];
        continue;
      }
      const TW* src = (i == r && r != j) ? jrow : xi;
      const TW f = src[t];
      // no test for f == 0: base - 0 * s is base for every finite s, and a
      // non-finite scaled pivot row has already marked the matrix singular;
      // the guarded form cost FP64 issue slots (20% of the panel time)
      for (int c = lane; c < nb; c += 32) {
        const TW base = (c == t) ? (TW)0 : src[c];
        xi[c] = base - f * srow[c];
      }
    }
    __syncthreads();  // the next column's candidates read the eliminated rows
  }
  // panel back to global memory
  for (int e = tid; e < (r1 - r0) * nb; e += kPanelThreads) {
    const int i = e / nb, t = e % nb;
    X[(int64_t)(r0 + i) * b + p + t] = P[i * ldp + t];
  }
  // the row exchanges of the panel, in order, on the columns outside it (each
  // CTA its share of those columns; they are not read during the panel)
  {
    const int nrest = b - nb;
    const int per = (nrest + CL - 1) / CL;
    const int c0 = q * per, c1 = min(nrest, c0 + per);
    for (int c = c0 + tid; c < c1; c += kPanelThreads) {
      const int cc = c < p ? c : c + nb;
      for (int t = 0; t < nb; ++t) {
        const int j = p + t, r = piv_hist[t];
        if (r != j) {
          const TW a = X[(int64_t)j * b + cc];
          X[(int64_t)j * b + cc] = X[(int64_t)r * b + cc];
          X[(int64_t)r * b + cc] = a;
        }
      }
    }
  }
  cluster.sync();  // every row exchange of the other columns is done
  // W = X[J, :] (the CUDA-core trailing update reads the pivot rows of the
  // other columns from W; the tensor-core one packs them from X itself, where
  // they stay unchanged until that pack)
  if (nb < b && !active_only) {
    TW* W = (TW*)d.wrow;
    const int64_t tot = (int64_t)nb * b;
    const int64_t per = (tot + CL - 1) / CL;
    const int64_t e0 = q * per, e1 = min(tot, e0 + per);
    for (int64_t e = e0 + tid; e < e1; e += kPanelThreads) {
      const int64_t tt = e / b, c = e % b;
      W[e] = X[(int64_t)(p + tt) * b + c];
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// X[:, rest] = T[:, J] * W[:, rest] + (rows of J ? 0 : X[:, rest]).
template <typename TW>
__global__ void __launch_bounds__(256) gj_update_kernel(const InvDesc* __restrict__ descs, int p, int nb) {
  using Cfg = TileCfg<TW>;
  using TG = TileGemm<TW, TW, TW, Cfg::BM, Cfg::BN, Cfg::BK, Cfg::TM, Cfg::TN>;
  __shared__ typename TG::Smem smem;
  const InvDesc d = descs[blockIdx.z];
  const int b = d.b;
  const int m0 = blockIdx.y * Cfg::BM, n0 = blockIdx.x * Cfg::BN;
  if (m0 >= b || n0 >= b) return;
  nb = min(nb, b - p);
  if (nb <= 0 || nb >= b) return;  // past this matrix's end, or its panel is the whole matrix
  if (n0 >= p && n0 + Cfg::BN <= p + nb) return;  // tile inside the panel
  TW* X = (TW*)d.work;
  TW acc[Cfg::TM][Cfg::TN];
#pragma unroll
  for (int i = 0; i < Cfg::TM; ++i)
#pragma unroll
    for (int j = 0; j < Cfg::TN; ++j) acc[i][j] = (TW)0;
  TG::run(smem, X + p, b, 0, (const TW*)d.wrow, b, 0, m0, n0, b, b, nb, acc);
  const int tx = threadIdx.x % TG::TX, ty = threadIdx.x / TG::TX;
#pragma unroll
  for (int i = 0; i < Cfg::TM; ++i) {
    const int r = m0 + ty * Cfg::TM + i;
    if (r >= b) continue;
    const bool in_j = (r >= p && r < p + nb);
#pragma unroll
    for (int j = 0; j < Cfg::TN; ++j) {
      const int c = n0 + tx * Cfg::TN + j;
      if (c >= b || (c >= p && c < p + nb)) continue;
      TW* x = X + (int64_t)r * b + c;
      *x = in_j ? acc[i][j] : (*x + acc[i][j]);
    }
  }
}

// Descriptors of the tensor-core trailing update of panel [p, p + nb): the
// panel columns T = X[:, J] as the left operand (by rows), the pivot rows
// W = X[J, :] as the right one (by columns; read in place: the panel left
// them there and nothing writes them before this pack), out = X with the rows
// of J taking no addend and the columns of J left alone.  A matrix past its last panel,
// or whose panel is the whole matrix, gets an empty problem.
__global__ void gj_tc_setup_kernel(const InvDesc* __restrict__ descs, int count, int p, int nb,
                                   oz::PackDesc* __restrict__ pa, oz::PackDesc* __restrict__ pb,
                                   oz::Problem* __restrict__ pr) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= count) return;
  const InvDesc d = descs[u];
  const int b = d.b;
  const int w = min(nb, b - p);
  const bool live = w > 0 && w < b;
  double* X = (double*)d.work;
  pa[u] = oz::PackDesc{X + (live ? p : 0), b, live ? b : 0, live ? w : 0, 0, u};
  pb[u] = oz::PackDesc{X + (live ? (int64_t)p * b : 0), b, live ? w : 0, live ? b : 0, 1, u};
  oz::Problem q{};
  q.a_slab = q.b_slab = u;
  q.cin = X;
  q.ldcin = b;
  q.out = X;
  q.ldo = b;
  q.m = q.n = live ? b : 0;
  q.nocin_r0 = q.skip_c0 = p;
  q.nocin_r1 = q.skip_c1 = p + (live ? w : 0);
  pr[u] = q;
}

// Descriptors of the product that completes the panel columns J = [p, p + w)
// of the rows already used as pivots, [0, p), which the panel kernel leaves
// alone (active_only): in Gauss-Jordan form every non-pivot row of the panel
// ends as -X_old[i, J] A^-1, with A^-1 = X[P, J] the pivot rows' panel
// columns after the panel, so
//     X[0:p, J] = -X[0:p, J] X[p:p+w, J]     (one digit product, K = w).
__global__ void gj_tc_done_setup_kernel(const InvDesc* __restrict__ descs, int count, int p, int nb,
                                        oz::PackDesc* __restrict__ pa, oz::PackDesc* __restrict__ pb,
                                        oz::Problem* __restrict__ pr) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= count) return;
  const InvDesc d = descs[u];
  const int b = d.b;
  const int w = min(nb, b - p);
  const bool live = p > 0 && w > 0;
  double* X = (double*)d.work;
  pa[u] = oz::PackDesc{X + (live ? p : 0), b, live ? p : 0, live ? w : 0, 0, u};
  pb[u] = oz::PackDesc{X + (live ? (int64_t)p * b + p : 0), b, live ? w : 0, live ? w : 0, 1, u};
  oz::Problem q{};
  q.a_slab = q.b_slab = u;
  q.cin = nullptr;
  q.out = X + (live ? p : 0);
  q.ldcin = q.ldo = b;
  q.m = live ? p : 0;
  q.n = live ? w : 0;
  pr[u] = q;
}

// Descriptors of a cross product inside a block of delayed panels
// J_0 = [p, p + nb), J_1, ... (see run_batch_t), for its panel J_i (i >= 1)
// and the earlier ones J_<i = [p, p + i nb):
//   dir 0 brings the columns of J_i up to date with the composite transform
//         of J_<i:  X[:, J_i] = X[:, J_<i] X[J_<i, J_i] + X[:, J_i];
//   dir 1 applies the transform of J_i to the columns of J_<i:
//         X[:, J_<i] = X[:, J_i] X[J_i, J_<i] + X[:, J_<i];
// the transform's own pivot rows take no addend.  A matrix without panel J_i
// gets an empty problem.
__global__ void gj_tc_cross_setup_kernel(const InvDesc* __restrict__ descs, int count, int p, int nb, int i, int dir,
                                         oz::PackDesc* __restrict__ pa, oz::PackDesc* __restrict__ pb,
                                         oz::Problem* __restrict__ pr) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= count) return;
  const InvDesc d = descs[u];
  const int b = d.b;
  const int wi = max(0, min(nb, b - p - i * nb));  // width of J_i in this matrix
  const int wl = max(0, min(i * nb, b - p));       // width of J_<i
  const bool live = wi > 0 && wl > 0;
  const int ca = dir ? p + i * nb : p, wa = dir ? wi : wl;  // the transform's columns (and pivot rows)
  const int cc = dir ? p : p + i * nb, wc = dir ? wl : wi;  // the columns brought up to date
  double* X = (double*)d.work;
  pa[u] = oz::PackDesc{X + (live ? ca : 0), b, live ? b : 0, live ? wa : 0, 0, u};
  pb[u] = oz::PackDesc{X + (live ? (int64_t)ca * b + cc : 0), b, live ? wa : 0, live ? wc : 0, 1, u};
  oz::Problem q{};
  q.a_slab = q.b_slab = u;
  q.cin = X + (live ? cc : 0);
  q.out = X + (live ? cc : 0);
  q.ldcin = q.ldo = b;
  q.m = live ? b : 0;
  q.n = live ? wc : 0;
  q.nocin_r0 = live ? ca : 0;
  q.nocin_r1 = live ? ca + wa : 0;
  pr[u] = q;
}

// Panels per block of delayed tensor-core updates (the code takes any S >= 2).
// Two: with four (K = 256) the trailing product's tiles lose the FP32 integer
// shortcut of K <= 128 and the cross products grow with the block; measured
// on the 64-block default step, 216.3 against 212.0 ms (and, with the
// two-pass digit-product kernel and the shortcut for any K, 208.9 against
// 205.5 ms).
int inv_delay(int, int) { return 2; }

struct TcLayout {
  int rpa, rpb, kpad;
  size_t da, db, ea, eb, pa, pb, pr, total;
};

TcLayout tc_layout(int bmax, int count) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  TcLayout L;
  L.rpa = (bmax + oz::tile_m() - 1) / oz::tile_m() * oz::tile_m();
  L.rpb = (bmax + oz::tile_n() - 1) / oz::tile_n() * oz::tile_n();
  // the inner length of the widest update is the width of a block of
  // delayed panels
  const int nb = inv_panel_width(bmax, F64, true);
  L.kpad = (std::min(inv_delay(bmax, nb) * nb, bmax) + oz::tile_k() - 1) / oz::tile_k() * oz::tile_k();
  const size_t K = L.kpad;
  size_t o = 0;
  L.da = o;
  o += al((size_t)count * oz::kDigits * L.rpa * K * 2);
  L.db = o;
  o += al((size_t)count * oz::kDigits * L.rpb * K * 2);
  L.ea = o;
  o += al((size_t)count * L.rpa * 4);
  L.eb = o;
  o += al((size_t)count * L.rpb * 4);
  L.pa = o;
  o += al((size_t)count * sizeof(oz::PackDesc));
  L.pb = o;
  o += al((size_t)count * sizeof(oz::PackDesc));
  L.pr = o;
  o += al((size_t)count * sizeof(oz::Problem));
  L.total = o;
  return L;
}

// The row interchanges perm[0..b) undone as column interchanges taken in
// reverse order: perm is overwritten with col_of, the source column of every
// output column (one CTA per matrix, once, instead of once per output CTA).
__global__ void gj_colperm_kernel(const InvDesc* __restrict__ descs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* col_of = (int*)smem_raw;
  const InvDesc d = descs[blockIdx.x];
  const int b = d.b;
  for (int c = threadIdx.x; c < b; c += blockDim.x) col_of[c] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = b - 1; j >= 0; --j) {
      const int q = d.perm[j];
      if (q != j) {
        const int a = col_of[j];
        col_of[j] = col_of[q];
        col_of[q] = a;
      }
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < b; c += blockDim.x) d.perm[c] = col_of[c];
}

// out[r][c] = X[r][col_of[c]] with col_of from gj_colperm_kernel (in perm).
template <typename TW, typename TO>
__global__ void gj_finalize_kernel(const InvDesc* __restrict__ descs, int rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* col_of = (int*)smem_raw;
  const InvDesc d = descs[blockIdx.y];
  const int b = d.b;
  for (int c = threadIdx.x; c < b; c += blockDim.x) col_of[c] = d.perm[c];
  __syncthreads();
  const TW* X = (const TW*)d.work;
  TO* out = (TO*)d.dst;
  const int r0 = blockIdx.x * rows_per_cta;
  const int r1 = min(b, r0 + rows_per_cta);
  for (int r = r0; r < r1; ++r)
    for (int c = threadIdx.x; c < b; c += blockDim.x) out[(int64_t)r * d.ldd + c] = (TO)X[(int64_t)r * b + col_of[c]];
}

template <typename TW>
cudaError_t run_batch_t(int in_dtype, int out_dtype, const InvDesc* d_desc, int count, int b, DevStatus* d_status,
                        cudaStream_t s, int* launches, const InvTc* tc, InvTiming* tm) {
  int nl = 0;
  zero_amax_kernel<<<(count + 127) / 128, 128, 0, s>>>(d_desc, count);
  ++nl;
  {
    const int64_t nel = (int64_t)b * b;
    const int chunks = (int)std::min<int64_t>(64, (nel + 255 * 8) / (256 * 8));
    dim3 g(std::max(chunks, 1), count);
    gj_init_kernel<TW><<<g, 256, 0, s>>>(d_desc, in_dtype);
    ++nl;
  }
  const int nb = inv_panel_width(b, sizeof(TW) == 8 ? F64 : F32, tc != nullptr);
  // cluster size: spread the panel over more SMs when few matrices are batched,
  // and keep a CTA's rows within about 72 KB so that three CTAs share an SM
  // (their per-column barriers and pivot exchanges then overlap one another's
  // eliminations: measured 18% less panel time than one 135 KB CTA per SM)
  // (m rows eliminated per matrix: b, or with tensor-core updates only the
  // b - p rows not yet used as pivots, so later panels take smaller clusters)
  // a tuned bias (mbinv_autotune) scales the heuristic's choice by 2^bias, up
  // to clusters of 16 CTAs (non-portable; only where the device can co-schedule
  // one, checked per launch) for the small, latency-bound batches
  const int bias = cluster_bias(b, count, sizeof(TW) == 8 ? F64 : F32, tc != nullptr);
  auto cluster_for = [&](int m) {
    int CL = 8;
    while (CL > 1 && count * CL > 2 * 152) CL >>= 1;
    // fewer, fuller CTAs while the smaller cluster still covers every SM
    while (CL > 1 && count * (CL / 2) >= 152 && (m + CL / 2 - 1) / (CL / 2) * (nb + 1) * sizeof(TW) <= 64 * 1024)
      CL >>= 1;
    while (CL < 8 && ((size_t)((m + CL - 1) / CL) + 4) * (nb + 1) * sizeof(TW) > 72 * 1024) CL <<= 1;
    for (int t = 0; t < bias && CL < 16; ++t) CL <<= 1;
    for (int t = 0; t < -bias && CL > 1; ++t) CL >>= 1;
    while (CL < 8 && ((size_t)((m + CL - 1) / CL) + 4) * (nb + 1) * sizeof(TW) > (size_t)kSmemLimit) CL <<= 1;
    return CL;
  };
  {
    const int CL = cluster_for(b);
    if (((size_t)((b + CL - 1) / CL) + 4) * (nb + 1) * sizeof(TW) > (size_t)kSmemLimit) return cudaErrorInvalidValue;
  }
  {
    cudaError_t e = once_per_device((const void*)gj_panel_kernel<TW>, [] {
      cudaError_t e2 = cudaFuncSetAttribute(gj_panel_kernel<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
      if (e2 != cudaSuccess) return e2;
      return cudaFuncSetAttribute(gj_panel_kernel<TW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    });
    if (e != cudaSuccess) return e;
  }
  // one panel factorisation [pp, pp + nb) of every matrix (event-timed when asked)
  auto panel = [&](int pp) -> cudaError_t {
    const int w = std::min(nb, b - pp);  // widest panel of this step (b is the largest order)
    const int m = tc && w < b ? b - pp : b;
    int CL = cluster_for(m);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    auto configure = [&]() {
      cfg.gridDim = dim3(count * CL, 1, 1);
      cfg.blockDim = dim3(kPanelThreads, 1, 1);
      cfg.dynamicSmemBytes = ((size_t)((m + CL - 1) / CL) + 4) * (w + 1) * sizeof(TW);
      cfg.stream = s;
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = CL;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
    };
    configure();
    if (CL > 8) {
      // a non-portable cluster: only if one can be resident at all
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, gj_panel_kernel<TW>, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();  // the query's error is not the call's
        CL = 8;
        configure();
      }
    }
    const bool timed = tm && tm->n + 2 <= tm->cap;
    if (timed) cudaEventRecord(tm->ev[tm->n], s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, gj_panel_kernel<TW>, d_desc, pp, w, d_status, tc && w < b ? 1 : 0);
    if (e != cudaSuccess) return e;
    if (timed) {
      cudaEventRecord(tm->ev[tm->n + 1], s);
      tm->n += 2;
    }
    ++nl;
    return cudaSuccess;
  };
  cudaError_t e;
  if (tc && nb < b) {
    // Tensor-core updates, delayed over blocks of S panels J_0 = [p, p + nb),
    // J_1, ..., J_{S-1} (S = inv_delay, two): the columns outside the block J receive
    // one rank-S nb update (K = S nb) instead of S rank-nb ones, which divides
    // the per-entry epilogues of the widest products by S.  The block's
    // columns carry the composite transform first; for i = 0 .. S-1:
    //   (i > 0) X[:, J_i]  += X[:, J_<i] X[J_<i, J_i]   (J_i up to date)
    //   panel J_i; rows done before J_i (product)
    //   (i > 0) X[:, J_<i] += X[:, J_i] X[J_i, J_<i]    (J_i's transform on J_<i)
    // then X[:, rest] += X[:, J] X[J, rest] (each "+=" with the rows of the
    // transform's own pivots taking no addend).  This is the sequence of
    // single-panel updates regrouped: the pivot rows X[J, rest] are untouched
    // (only exchanged) until the last product.
    const TcLayout T = tc_layout(b, count);
    char* base = (char*)tc->scratch;
    auto* pa = (oz::PackDesc*)(base + T.pa);
    auto* pb = (oz::PackDesc*)(base + T.pb);
    auto* pr = (oz::Problem*)(base + T.pr);
    auto* da = (__nv_bfloat16*)(base + T.da);
    auto* db = (__nv_bfloat16*)(base + T.db);
    int* ea = (int*)(base + T.ea);
    int* eb = (int*)(base + T.eb);
    oz::Params Q{};
    Q.kb0 = 0;
    Q.ea = ea;
    Q.eb = eb;
    Q.ea_rows = T.rpa;
    Q.eb_rows = T.rpb;
    Q.err = tc->err;
    Q.coprime_grid = 1;  // the skipped panel columns recur every tiles_n tiles
    // one grouped digit product over K = kpad (a multiple of 64, at most T.kpad)
    auto product = [&](int kpad, double alpha, double beta, int tiles_m, int tiles_n) -> cudaError_t {
      cudaError_t e2 = oz::launch_pack2(oz::PackSet{pa, count, T.rpa, da, ea}, oz::PackSet{pb, count, T.rpb, db, eb},
                                        kpad, s);
      if (e2 != cudaSuccess) return e2;
      Q.kpad = kpad;
      Q.nkb = kpad / oz::tile_k();
      Q.alpha = alpha;
      Q.beta = beta;
      Q.tiles_m = tiles_m;
      Q.tiles_n = tiles_n;
      nl += 2;
      return oz::launch_gemm(da, count, T.rpa, db, count, T.rpb, Q, pr, count, s);
    };
    auto kround = [](int x) { return (x + oz::tile_k() - 1) / oz::tile_k() * oz::tile_k(); };
    const int k1 = kround(nb);
    const int S = inv_delay(b, nb);
    const int g = (count + 127) / 128;
    // rows [0, pp) of the panel [pp, pp + nb): p x nb outputs per matrix
    auto done = [&](int pp) -> cudaError_t {
      if (pp == 0) return cudaSuccess;
      gj_tc_done_setup_kernel<<<g, 128, 0, s>>>(d_desc, count, pp, nb, pa, pb, pr);
      ++nl;
      return product(k1, -1.0, 0.0, (pp + oz::tile_m() - 1) / oz::tile_m(), (nb + oz::tile_n() - 1) / oz::tile_n());
    };
    auto cross = [&](int pp, int i, int dir) -> cudaError_t {
      gj_tc_cross_setup_kernel<<<g, 128, 0, s>>>(d_desc, count, pp, nb, i, dir, pa, pb, pr);
      ++nl;
      const int wl = std::min(i * nb, b - pp);  // J_<i of the largest matrix
      if (dir == 0) return product(kround(wl), 1.0, 1.0, T.rpa / oz::tile_m(), (nb + oz::tile_n() - 1) / oz::tile_n());
      return product(k1, 1.0, 1.0, T.rpa / oz::tile_m(), (wl + oz::tile_n() - 1) / oz::tile_n());
    };
    for (int p = 0; p < b; p += S * nb) {
      for (int i = 0; i < S && p + i * nb < b; ++i) {
        const int pi = p + i * nb;
        if (i > 0 && (e = cross(p, i, 0)) != cudaSuccess) return e;
        if ((e = panel(pi)) != cudaSuccess) return e;
        if ((e = done(pi)) != cudaSuccess) return e;
        if (i > 0 && (e = cross(p, i, 1)) != cudaSuccess) return e;
      }
      gj_tc_setup_kernel<<<g, 128, 0, s>>>(d_desc, count, p, S * nb, pa, pb, pr);
      ++nl;
      const int kt = kround(std::min(S * nb, b - p));
      if ((e = product(kt, 1.0, 1.0, T.rpa / oz::tile_m(), T.rpb / oz::tile_n())) != cudaSuccess) return e;
    }
  } else {
    for (int p = 0; p < b; p += nb) {
      if ((e = panel(p)) != cudaSuccess) return e;
      const int w = std::min(nb, b - p);
      if (w < b) {  // matrices whose panel is not the whole matrix need the trailing update
        using Cfg = TileCfg<TW>;
        dim3 g((b + Cfg::BN - 1) / Cfg::BN, (b + Cfg::BM - 1) / Cfg::BM, count);
        gj_update_kernel<TW><<<g, 256, 0, s>>>(d_desc, p, w);
        ++nl;
      }
    }
  }
  {
    const int rows = 8;
    dim3 g((b + rows - 1) / rows, count);
    const size_t sm = (size_t)b * sizeof(int);
    gj_colperm_kernel<<<count, 128, sm, s>>>(d_desc);
    ++nl;
    if (out_dtype == F64)
      gj_finalize_kernel<TW, double><<<g, 256, sm, s>>>(d_desc, rows);
    else
      gj_finalize_kernel<TW, float><<<g, 256, sm, s>>>(d_desc, rows);
    ++nl;
  }
  if (launches) *launches += nl;
  return cudaGetLastError();
}

}  // namespace

int inv_panel_width(int b, int wtype, bool tc) {
  const size_t es = wtype == F64 ? 8 : 4;
  if (b <= kMaxPanelWidth && (size_t)b * (b + 1) * es <= 132 * 1024) return b;  // whole matrix in one panel
  // the tensor-core update takes K in blocks of 64; wider panels must still
  // fit a cluster of 8 CTAs
  if (tc && wtype == F64 && ((size_t)(b + 7) / 8 + 4) * 65 * es <= (size_t)kSmemLimit) return 64;
  return 32;
}

size_t inv_tc_bytes(int bmax, int count) { return tc_layout(bmax, count).total; }

void inv_flop_split(int b, int wtype, bool tc, double* panel_flops, double* update_flops) {
  const int nb = inv_panel_width(b, wtype, tc);
  double pf = 0, uf = 0;
  for (int p = 0; p < b; p += nb) {
    const double w = std::min(nb, b - p);
    // with tensor-core updates a panel eliminates only the rows not yet used
    // as pivots; the others' panel columns come from a product
    const double rows = (tc && w < b) ? b - p : b;
    pf += 2.0 * rows * w * w;
    uf += 2.0 * b * w * (b - w) + 2.0 * (b - rows) * w * w;
  }
  *panel_flops = pf;
  *update_flops = uf;
}

namespace {
std::mutex g_bias_mu;
std::map<std::tuple<int, int, int, int>, int> g_bias;  // (b, count bucket, wtype, tc) -> bias
int count_bucket(int count) {
  int q = 1;
  while (q < count) q <<= 1;
  return q;
}
}  // namespace

void set_cluster_bias(int b, int count, int wtype, bool tc, int bias) {
  std::lock_guard<std::mutex> lock(g_bias_mu);
  g_bias[std::make_tuple(b, count_bucket(count), wtype, (int)tc)] = bias;
}

int cluster_bias(int b, int count, int wtype, bool tc) {
  std::lock_guard<std::mutex> lock(g_bias_mu);
  auto it = g_bias.find(std::make_tuple(b, count_bucket(count), wtype, (int)tc));
  return it == g_bias.end() ? 0 : it->second;
}

cudaError_t run_inverse_batch(int in_dtype, int out_dtype, int wtype, const InvDesc* d_desc, int count, int b,
                              DevStatus* d_status, cudaStream_t s, int* launches, const InvTc* tc,
                              InvTiming* timing) {
  if (count <= 0) return cudaSuccess;
  if (wtype == F64) return run_batch_t<double>(in_dtype, out_dtype, d_desc, count, b, d_status, s, launches, tc, timing);
  if (tc) return cudaErrorInvalidValue;
  return run_batch_t<float>(in_dtype, out_dtype, d_desc, count, b, d_status, s, launches, nullptr, timing);
}

}  // namespace mbinv

namespace mbinv {
namespace {

template <typename TS>
__device__ double colsum_max(const TS* a, int64_t ld, int b) {
  double m = 0.0;
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < b; ++r) s += fabs((double)a[(int64_t)r * ld + c]);
    m = s > m ? s : m;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  __syncthreads();
  return m;  // valid in thread 0
}

// One CTA per matrix: ||src||_1 ||dst||_1 (largest column sums), folded
// into d.cond as the bit pattern of a non-negative double (NaN stays out:
// a singular inverse is reported through the status word instead).
__global__ void __launch_bounds__(1024) cond1_kernel(const InvDesc* __restrict__ descs, int in_dtype,
                                                     int out_dtype) {
  const InvDesc d = descs[blockIdx.x];
  if (!d.cond) return;
  const double a = in_dtype == F64 ? colsum_max((const double*)d.src, d.lds, d.b)
                                   : colsum_max((const float*)d.src, d.lds, d.b);
  const double x = out_dtype == F64 ? colsum_max((const double*)d.dst, d.ldd, d.b)
                                    : colsum_max((const float*)d.dst, d.ldd, d.b);
  if (threadIdx.x == 0) {
    const double k = a * x;
    if (k >= 0.0 && k <= 1.7976931348623157e308) atomicMax(d.cond, (unsigned long long)__double_as_longlong(k));
  }
}

}  // namespace

cudaError_t launch_cond1(const InvDesc* d_desc, int count, int in_dtype, int out_dtype, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  cond1_kernel<<<count, 1024, 0, s>>>(d_desc, in_dtype, out_dtype);
  return cudaGetLastError();
}

}  // namespace mbinv
