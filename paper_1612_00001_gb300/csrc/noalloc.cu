// mbinv_invert_noalloc: one b x b inverse (the library's pivoted Gauss-Jordan
// kernels) whose scratch lives in a fixed device array instead of memory
// allocated per call.
//
// Who needs it: callers that must not allocate device memory at the moment
// they invert - code running while a framework's caching allocator already
// holds (nearly) all of the GPU's memory, code that must not trigger the
// implicit device-wide synchronisation of cudaFree, and latency-critical
// loops that cannot afford an allocation per call.  They pass the input and
// the output; everything else the kernels need (descriptor, status word,
// pivot record, FP64 working copy, pivot-row buffer) sits in g_scratch.
//
// Rules of use
//   - b <= MBINV_NOALLOC_MAX_B (512); larger b is refused with MBINV_EINVAL
//     before anything is launched.
//   - g_scratch is one array per device, shared by every call on that device
//     and kept between calls (each call rewrites every word it reads).  Calls
//     whose work overlaps on the GPU - two host threads, or two streams -
//     race on it; serialise them.
//   - Each call waits on the host for its own result (it reads its status
//     word back before returning).
//   - The first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; that first call
//     should come before any stream capture.
//   - No cudaMalloc, cudaFree or other allocating routine is called.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include "../../include/mbinv.h"
#include "mbinv_internal.h"

namespace mbinv {
namespace {

constexpr int kMaxB = MBINV_NOALLOC_MAX_B;
constexpr size_t kDescOff = 0;       // InvDesc
constexpr size_t kStatusOff = 256;   // DevStatus
constexpr size_t kAmaxOff = 512;     // max |entry|
constexpr size_t kPermOff = 768;     // kMaxB ints
constexpr size_t kWorkOff = kPermOff + ((kMaxB * 4 + 255) / 256) * 256;
constexpr size_t kWrowOff = kWorkOff + (size_t)kMaxB * kMaxB * 8;
constexpr size_t kScratchBytes = kWrowOff + (size_t)32 * kMaxB * 8;  // about 2.2 MB

// Host code sees a stand-in for this symbol, not its device address: the
// address comes from cudaGetSymbolAddress (set-up below).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[128] = {};

// Writes the descriptor and resets the status word (no host copy needed).
__global__ void noalloc_setup_kernel(unsigned char* base, InvDesc d) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *(InvDesc*)(base + kDescOff) = d;
    DevStatus* st = (DevStatus*)(base + kStatusOff);
    st->singular = 0;
    st->tag = INT_MAX;
  }
}

}  // namespace
}  // namespace mbinv

extern "C" mbinv_status mbinv_invert_noalloc(const void* A, int64_t lda, void* X, int64_t ldx, int64_t b, int dtype,
                                             void* stream) {
  using namespace mbinv;
  if (!A || !X || b <= 0 || lda < b || ldx < b || (dtype != F64 && dtype != F32)) return MBINV_EINVAL;
  if (b > kMaxB) return MBINV_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return MBINV_ECUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return MBINV_ECUDA;
      g_addr[dev] = p;
    }
    base = (unsigned char*)g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  InvDesc d{};
  d.src = A;
  d.lds = lda;
  d.dst = X;
  d.ldd = ldx;
  d.work = base + kWorkOff;
  d.wrow = base + kWrowOff;
  d.perm = (int*)(base + kPermOff);
  d.amax = (unsigned long long*)(base + kAmaxOff);
  d.b = (int)b;
  d.tag = 0;
  noalloc_setup_kernel<<<1, 32, 0, s>>>(base, d);
  if (cudaGetLastError() != cudaSuccess) return MBINV_ECUDA;
  int launches = 0;
  if (run_inverse_batch(dtype, dtype, F64, (const InvDesc*)(base + kDescOff), 1, (int)b,
                        (DevStatus*)(base + kStatusOff), s, &launches) != cudaSuccess)
    return MBINV_ECUDA;
  DevStatus st{};
  if (cudaMemcpyAsync(&st, base + kStatusOff, sizeof st, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MBINV_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MBINV_ECUDA;
  return st.singular ? MBINV_ESINGULAR : MBINV_OK;
}
