// Internal declarations of the structured-operator library (host side).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fm.h"

namespace fm {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
void clear_error();

#define FM_TRY(expr)                          \
  do {                                        \
    fm_status _s = (expr);                    \
    if (_s != FM_OK) return _s;               \
  } while (0)

#define FM_CUDA(expr)                                                             \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      ::fm::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,                  \
                      cudaGetErrorString(_e));                                    \
      return _e == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA;          \
    }                                                                             \
  } while (0)

// Every kernel launch of the library goes through this counter.
extern std::atomic<uint64_t> g_launches;
inline fm_status after_launch(const char* what) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
    return FM_ERR_CUDA;
  }
  return FM_OK;
}

// Launch that lets the kernel's CTAs become resident while the previous kernel of the stream
// drains its last wave (programmatic dependent launch).  A kernel launched this way executes
// pdl_wait() (fm_device.cuh) before its first global-memory access, which returns once the
// previous grid has completed and its writes are visible; launched without the attribute,
// pdl_wait() returns at once.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}
// Launch tracing (trace.cu): while fm_trace_begin is in effect, trace_open records a start
// event on the launch's stream (returns its slot, or -1) and trace_close the end event.
extern std::atomic<int> g_trace_on;
int trace_open(cudaStream_t st);
void trace_close(int slot, cudaStream_t st, const char* name);

template <typename... KArgs, typename... Args>
inline fm_status pdl_go(const char* what, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                        cudaStream_t st, Args... args) {
  const int ts = g_trace_on.load(std::memory_order_relaxed) ? trace_open(st) : -1;
  cudaError_t e = launch_pdl(kern, grid, block, smem, st, args...);
  if (ts >= 0) trace_close(ts, st, what);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
    return FM_ERR_CUDA;
  }
  return after_launch(what);
}

// ------------------------------------------------------------------ dtypes
inline bool is_complex(fm_dtype d) { return d == FM_C64 || d == FM_C128; }
inline bool is_double(fm_dtype d) { return d == FM_F64 || d == FM_C128; }
inline int dtype_size(fm_dtype d) {
  switch (d) {
    case FM_I8: return 1;
    case FM_I32: return 4;
    case FM_F32: return 4;
    case FM_F64: return 8;
    case FM_C64: return 8;
    case FM_C128: return 16;
  }
  return 0;
}
inline fm_dtype real_of(fm_dtype d) {
  if (d == FM_C64) return FM_F32;
  if (d == FM_C128) return FM_F64;
  return d;
}
inline fm_dtype complex_of(fm_dtype d) {
  if (d == FM_F32) return FM_C64;
  if (d == FM_F64) return FM_C128;
  return d;
}

// ------------------------------------------------------------------ per-device tables
// W_{kTwMax}^m = exp(-2 pi i m / kTwMax), m in [0, kTwMax), in FP32 and FP64, computed once
// per device in FP64 with sincospi.
constexpr int kTwLog = 14;
constexpr int kTwMax = 1 << kTwLog;
struct DeviceTables {
  float2* tw32 = nullptr;
  double2* tw64 = nullptr;
  float2* twp32 = nullptr;   // pass-twiddle tables of the Stockham passes (fm_device.cuh)
  double2* twp64 = nullptr;
};
fm_status device_tables(int device, DeviceTables** out);
// The tables of `device` if they exist already, else nullptr (never allocates).
DeviceTables* device_tables_if_ready(int device);

// Dense product y = M x (adj: M^H x) of a leaf with fm_set_dense on, complex columns of one
// precision (dense.cu).
fm_status dense_apply(const fm_op_s* A, bool adj, const void* in, int64_t ldi, void* out, int64_t ldo,
                      int64_t ncols, bool dbl, int beta, cudaStream_t st);

// Look up (and so reserve) the static scratch of fm_circulant_apply_noalloc on `device`, the
// current device; called when a Circulant operator is built there (noalloc.cu).
fm_status noalloc_prepare(int device);

// ------------------------------------------------------------------ operators
enum OpKind {
  K_FOURIER, K_CIRCULANT, K_TOEPLITZ, K_HADAMARD, K_DIAG, K_PARTIAL,
  K_PRODUCT, K_SUM, K_BLKDIAG, K_KRON, K_HERMITIAN, K_BLOCKS
};

// Twiddles and spectra for a length-L transform done in two passes (L = N1 * N2): every
// transform longer than one tile, and (Fourier, Circulant) small FP64 problems of
// 2^11 .. 2^13, spread over more CTAs.
constexpr int64_t kBigPlanMin = 2048;
struct BigPlan {
  int64_t L = 0, N1 = 0, N2 = 0;
  float2* tw32 = nullptr;   // W_L^m, m in [0, L)
  double2* tw64 = nullptr;
};

struct Workspace {
  std::mutex mu;
  void* ptr = nullptr;
  size_t bytes = 0;
  int device = -1;
};

}  // namespace fm

struct fm_op_s {
  std::atomic<int> refs{1};
  fm::OpKind kind;
  int64_t rows = 0, cols = 0;
  bool real = true;
  int device = 0;
  // leaf parameters
  int ortho = 0;                 // Fourier
  int log2n = 0;                 // Hadamard
  fm_had_mode had_mode = FM_HAD_FP32;
  int64_t L = 0;                 // transform length (Fourier n, circulant n, Toeplitz embedding)
  // circulant / Toeplitz spectrum of the embedding, already divided by L
  // (natural order, and the row-permuted copy used by the two-pass plan)
  double2* spec64 = nullptr;
  float2* spec32 = nullptr;
  double2* spec64_perm = nullptr;
  float2* spec32_perm = nullptr;
  double cap = 0.0;              // max |spectrum * L|^2 (FISTA step cap)
  // diagonal
  double2* d64 = nullptr;        // complex diagonal (both precisions) ...
  float2* d32 = nullptr;
  double* dr64 = nullptr;        // ... or real diagonal
  float* dr32 = nullptr;
  // row selection
  int32_t* idx = nullptr;        // m selected rows
  int32_t* inv = nullptr;        // n entries: r if idx[r] == j, else -1
  std::vector<int32_t> idx_host;
  // two-pass plan for long transforms
  fm::BigPlan big;
  // execution plan of the tile transforms (fm_set_plan / fm_calibrate): tile shape of strided
  // views (0 automatic, 1 default tile, 2 wide tile, 3 wide tile in 4 groups) and radix cap (0
  // schedule table, 3 radix <= 8)
  int tile = 0, rcap = 0;
  // dense execution of a small leaf (fm_set_dense): the matrix, column-major rows x cols
  int dense = 0;
  float2* m32 = nullptr;
  double2* m64 = nullptr;
  // composites (Blocks: kids[i * blk_c + j] is block (i, j) of a blk_r x blk_c grid)
  std::vector<fm_op_s*> kids;
  int blk_r = 0, blk_c = 0;
  fm::Workspace ws;
};

namespace fm {
void op_retain(fm_op_s* A);
void op_release(fm_op_s* A);
}  // namespace fm
