// Circulant transform that allocates no device memory.
//
// Some callers cannot allocate device memory when they apply an operator: programs whose
// device memory is owned by another allocator (a framework's caching allocator, or a
// fixed memory budget set at start-up), and code that must not trigger the implicit
// device-wide synchronisation of cudaMalloc / cudaFree.  fm_forward / fm_backward grow a
// per-operator workspace on demand, which such callers cannot allow.  This entry point
// applies a Circulant operator to complex64 columns with the scratch of the two-pass
// plan (long transforms, n > 16384) taken from a fixed array that lives in the library's
// device image instead: it is reserved on a device when the first Circulant operator is
// built there and held until the process exits.  The operator itself is built beforehand
// with fm_circulant, which does allocate.
#include <mutex>

#include "exec.h"

namespace fm {

// 16 MiB: n * ncols * 8 bytes of two-pass scratch, e.g. n = 2^18 with 8 columns per call.
constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocScratchBytes / sizeof(float2)];

// Device address of g_noalloc_scratch per device.  The library's device code is loaded
// lazily, so looking the address up is what loads this array's module and reserves its
// 16 MiB on the device: fm_circulant does it (construction allocates anyway), and the
// entry point below only reads the cached value.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

fm_status noalloc_prepare(int dev) {
  if (dev < 0 || dev >= 64) { set_error("device %d out of range", dev); return FM_ERR_INVALID_ARG; }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  g_noalloc_ptr[dev] = p;
  return FM_OK;
}

static void* noalloc_scratch(int dev) {
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  return g_noalloc_ptr[dev];
}

}  // namespace fm

using namespace fm;

extern "C" fm_status fm_circulant_apply_noalloc(fm_op C, int adjoint, const void* X, int64_t ldx, void* Y,
                                                int64_t ldy, int64_t ncols, void* stream) {
  clear_error();
  if (!C) { set_error("null operator"); return FM_ERR_INVALID_ARG; }
  if (C->kind != K_CIRCULANT) { set_error("fm_circulant_apply_noalloc takes a Circulant operator"); return FM_ERR_INVALID_ARG; }
  if (ncols < 0) { set_error("ncols < 0"); return FM_ERR_INVALID_ARG; }
  if (ncols == 0) return FM_OK;
  if (!X || !Y) { set_error("null data pointer"); return FM_ERR_INVALID_ARG; }
  const int64_t n = C->rows;
  if (ldx < n || ldy < n) { set_error("leading dimension smaller than n"); return FM_ERR_SHAPE; }
  const size_t xb = (size_t)((ncols - 1) * ldx + n) * sizeof(float2);
  const size_t yb = (size_t)((ncols - 1) * ldy + n) * sizeof(float2);
  const char* xp = (const char*)X;
  const char* yp = (const char*)Y;
  if (xp < yp + yb && yp < xp + xb) { set_error("output overlaps input"); return FM_ERR_ALIAS; }
  int dev = 0;
  FM_CUDA(cudaGetDevice(&dev));
  if (dev != C->device) { set_error("operator lives on device %d, current is %d", C->device, dev); return FM_ERR_INVALID_ARG; }
  Ctx ctx;
  ctx.st = (cudaStream_t)stream;
  ctx.tabs = device_tables_if_ready(dev);
  if (!ctx.tabs) { set_error("build the operator on this device first"); return FM_ERR_INVALID_ARG; }
  View in, out;
  in.p = (void*)X;
  in.dt = FM_C64;
  in.ld = ldx;
  in.n = in.ostride = n;
  out.p = Y;
  out.dt = FM_C64;
  out.ld = ldy;
  out.n = out.ostride = n;
  // measure the scratch this call needs, without launching anything
  ctx.dry = true;
  FM_TRY(exec(C, adjoint != 0, in, out, ncols, 0, ctx));
  if (ctx.peak > kNoallocScratchBytes) {
    set_error("this call needs %zu bytes of scratch but the static scratch holds %zu: pass fewer columns per call",
              ctx.peak, kNoallocScratchBytes);
    return FM_ERR_UNSUPPORTED;
  }
  void* scratch = noalloc_scratch(dev);
  if (!scratch) { set_error("the static scratch of device %d is not set up: build the operator there", dev); return FM_ERR_INVALID_ARG; }
  ctx.dry = false;
  ctx.base = (char*)scratch;
  ctx.cap = kNoallocScratchBytes;
  ctx.used = 0;
  ctx.peak = 0;
  return exec(C, adjoint != 0, in, out, ncols, 0, ctx);
}
