// Launch tracing: the device time of every kernel the library launches, for profiling.
//
// While tracing is on, each launch is bracketed by two CUDA events recorded on the launch's
// stream (launch_pdl's callers and the FISTA launches call trace_open / trace_close).  An
// event between two kernels of a stream ends the early start that programmatic dependent
// launch gives the second one, so traced kernels run strictly one after another.
#include <cstring>
#include <mutex>
#include <vector>

#include "fm_internal.h"

namespace fm {

std::atomic<int> g_trace_on{0};

namespace {
struct TraceRec {
  cudaEvent_t a = nullptr, b = nullptr;
  char name[64] = {0};
};
std::mutex g_trace_mu;
std::vector<TraceRec> g_trace;  // pre-created event pairs
int g_trace_used = 0;
int g_trace_seen = 0;

void trace_free() {
  for (auto& r : g_trace) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  g_trace.clear();
  g_trace_used = 0;
  g_trace_seen = 0;
}
}  // namespace

int trace_open(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  ++g_trace_seen;
  if (!g_trace_on.load() || g_trace_used >= (int)g_trace.size()) return -1;
  const int slot = g_trace_used++;
  if (cudaEventRecord(g_trace[slot].a, st) != cudaSuccess) {
    (void)cudaGetLastError();
    g_trace_used--;
    return -1;
  }
  return slot;
}

void trace_close(int slot, cudaStream_t st, const char* name) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (slot >= (int)g_trace.size()) return;
  std::strncpy(g_trace[slot].name, name, sizeof(g_trace[slot].name) - 1);
  if (cudaEventRecord(g_trace[slot].b, st) != cudaSuccess) (void)cudaGetLastError();
}

}  // namespace fm

using namespace fm;

extern "C" fm_status fm_trace_begin(int32_t max_launches) {
  clear_error();
  if (max_launches < 1 || max_launches > (1 << 20)) { set_error("max_launches in [1, 2^20]"); return FM_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (g_trace_on.load()) { set_error("tracing is already on"); return FM_ERR_INVALID_ARG; }
  trace_free();
  g_trace.resize(max_launches);
  for (auto& r : g_trace) {
    cudaError_t e = cudaEventCreate(&r.a);
    if (e == cudaSuccess) e = cudaEventCreate(&r.b);
    if (e != cudaSuccess) {
      set_error("fm_trace_begin: %s", cudaGetErrorString(e));
      trace_free();
      return FM_ERR_CUDA;
    }
  }
  g_trace_on.store(1);
  return FM_OK;
}

extern "C" fm_status fm_trace_end(fm_trace_entry* out, int32_t max_entries, int32_t* n_entries) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (!g_trace_on.load()) { set_error("tracing is not on"); return FM_ERR_INVALID_ARG; }
  g_trace_on.store(0);
  fm_status s = FM_OK;
  const int n = g_trace_used;
  for (int i = 0; i < n; ++i) {
    float ms = -1.f;
    cudaError_t e = cudaEventSynchronize(g_trace[i].b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, g_trace[i].a, g_trace[i].b);
    if (e != cudaSuccess) {
      set_error("fm_trace_end: %s", cudaGetErrorString(e));
      s = FM_ERR_CUDA;
      break;
    }
    if (out && i < max_entries) {
      std::memcpy(out[i].kernel, g_trace[i].name, sizeof(out[i].kernel));
      out[i].ms = ms;
    }
  }
  if (n_entries) *n_entries = g_trace_seen;
  trace_free();
  return s;
}
