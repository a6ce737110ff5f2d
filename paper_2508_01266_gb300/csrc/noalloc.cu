// Jacobian product that allocates no device memory.
//
// lrcc_jacobian_apply stages the vectors and its per-vector scratch in buffers it
// allocates with cudaMalloc on first use.  Some callers cannot let a library
// allocate at call time: host applications that own the device allocator and forbid
// allocations from plug-ins, and latency-critical loops where cudaMalloc's implicit
// synchronization is not acceptable.  This entry point runs the same op list with
// the staging vectors and the scratch placed in one file-scope __device__ array of
// fixed size (kNoAllocElems complex128 elements, 64 MiB), which every GPU that loads
// the library keeps until the process exits.  The problem's fixed data and W-block
// workspace were allocated by lrcc_create / lrcc_set_ground_state beforehand.
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/lrcc.h"
#include "runtime.h"

namespace {

constexpr long long kNoAllocElems = 4LL << 20;  // complex128 elements (64 MiB)
constexpr int kMaxDevices = 64;

__device__ __align__(256) double2 g_noalloc_scratch[kNoAllocElems];

// Device address of g_noalloc_scratch per device, with the CUDA context it was looked up
// in: a new context on that device (after cudaDeviceReset, for example) has its own copy
// of the array, so the address is looked up again.
struct ScratchAddr {
  void* ctx = nullptr;
  double2* ptr = nullptr;
};
ScratchAddr g_noalloc_addr[kMaxDevices];
std::mutex g_noalloc_mu;

// cuCtxGetCurrent through the runtime's driver entry-point query (no link against libcuda).
typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = []() -> CtxGetCurrentFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return (CtxGetCurrentFn)f;
  }();
  return fn;
}

}  // namespace

extern "C" lrcc_status lrcc_jacobian_apply_noalloc(lrcc_problem* p, int32_t transpose, const void* x1,
                                                   const void* x2, void* y1, void* y2, void* stream) {
  if (!p) return LRCC_EINVAL;
  lrcc::Runtime& rt = p->rt;
  if (!p->have_t) {
    rt.err = "jacobian_apply_noalloc: ground state not set";
    return LRCC_EINVAL;
  }
  if (!x1 || !x2 || !y1 || !y2 || (transpose != 0 && transpose != 1)) {
    rt.err = "jacobian_apply_noalloc: bad arguments";
    return LRCC_EINVAL;
  }
  const lrcc::Plan& P = rt.plan;
  const long long vin = P.arena_size[lrcc::AR_IN], vscr = P.arena_size[lrcc::AR_SCR];
  const long long need = 2 * vin + vscr;
  if (need > kNoAllocElems) {
    rt.err = "jacobian_apply_noalloc: this problem needs " + std::to_string(need) +
             " complex128 elements of scratch; the static limit is " + std::to_string(kNoAllocElems) +
             " (64 MiB); use lrcc_jacobian_apply";
    return LRCC_EUNSUPPORTED;
  }
  int dev = 0;
  if (!rt.ck(cudaGetDevice(&dev), "jacobian_apply_noalloc: cudaGetDevice")) return LRCC_ECUDA;
  if (dev != rt.device) {
    rt.err = "jacobian_apply_noalloc: device " + std::to_string(dev) + " is current, but the problem's buffers " +
             "are on device " + std::to_string(rt.device) + "; make that device current";
    return LRCC_EINVAL;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    rt.err = "jacobian_apply_noalloc: device ordinal out of range";
    return LRCC_EUNSUPPORTED;
  }
  double2* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    void* ctx = nullptr;
    if (CtxGetCurrentFn f = ctx_get_current()) f(&ctx);
    ScratchAddr& a = g_noalloc_addr[dev];
    if (!a.ptr || ctx != a.ctx) {
      void* addr = nullptr;
      // host code must not use the symbol itself: ask the runtime for its device address
      if (!rt.ck(cudaGetSymbolAddress(&addr, g_noalloc_scratch), "jacobian_apply_noalloc: cudaGetSymbolAddress"))
        return LRCC_ECUDA;
      a.ptr = (double2*)addr;
      a.ctx = ctx;
    }
    base = a.ptr;
  }
  // a null handle is the caller's legacy default stream (this library is built with
  // per-thread default streams, under which 0 would name the calling thread's stream)
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamLegacy;
  double2* in = base;
  double2* out = base + vin;
  double2* scr = base + 2 * vin;
  double2* src = transpose ? out : in;
  double2* res = transpose ? in : out;
  const int nk = rt.dims.nk, o = rt.dims.nocc, v = rt.dims.nvir;
  const size_t b1 = (size_t)nk * o * v * sizeof(double2);
  const size_t b2 = (size_t)nk * nk * nk * o * o * v * v * sizeof(double2);
  // the array keeps the previous call's contents: the result side and the scratch
  // must start at zero because every op accumulates
  if (!rt.ck(cudaMemcpyAsync(src + P.off_x1, x1, b1, cudaMemcpyDeviceToDevice, st), "noalloc copy x1") ||
      !rt.ck(cudaMemcpyAsync(src + P.off_x2, x2, b2, cudaMemcpyDeviceToDevice, st), "noalloc copy x2") ||
      !rt.ck(cudaMemsetAsync(res, 0, (size_t)vin * sizeof(double2), st), "noalloc memset") ||
      (vscr > 0 && !rt.ck(cudaMemsetAsync(scr, 0, (size_t)vscr * sizeof(double2), st), "noalloc memset")))
    return LRCC_ECUDA;
  double2* ar[lrcc::AR_COUNT] = {rt.fix, in, out, scr, rt.ws};
  const bool prof = rt.prof;
  rt.prof = false;     // per-op event timing would create events
  rt.no_split = true;  // split-K partials would need a buffer
  lrcc_status s = rt.run(transpose ? rt.jacT : P.jac, ar, 1, st);
  rt.prof = prof;
  rt.no_split = false;
  if (s != LRCC_OK) return s;
  if (!rt.ck(cudaMemcpyAsync(y1, res + P.off_x1, b1, cudaMemcpyDeviceToDevice, st), "noalloc copy y1") ||
      !rt.ck(cudaMemcpyAsync(y2, res + P.off_x2, b2, cudaMemcpyDeviceToDevice, st), "noalloc copy y2"))
    return LRCC_ECUDA;
  return LRCC_OK;
}
