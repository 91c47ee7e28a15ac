// Execution of operator trees (exec.cu).
#pragma once

#include "fm_internal.h"

namespace fm {

// A block of columns seen as [ncols][outer][n][inner]: element (c, o, t, i) is at
// p + c*ld + o*ostride + t*inner + i (in elements of dt).
struct View {
  void* p = nullptr;
  fm_dtype dt = FM_C64;
  int64_t ld = 0, outer = 1, ostride = 0, n = 0, inner = 1;
};

// Workspace arena: a dry run measures the peak, the real run bump-allocates.
struct Ctx {
  cudaStream_t st = nullptr;
  bool dry = false;
  char* base = nullptr;
  size_t used = 0, peak = 0, cap = 0;
  DeviceTables* tabs = nullptr;
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    void* r = dry ? nullptr : (void*)(base + used);
    used += bytes;
    if (used > peak) peak = used;
    return r;
  }
};

fm_status natural_out_dtype(const fm_op_s* A, fm_dtype in, fm_dtype* out);
fm_status exec(const fm_op_s* A, bool adj, const View& in, const View& out, int64_t ncols, int beta, Ctx& ctx);

// Unscaled DFT of length L (dir -1: F, +1: F^H) of ncols packed columns, times `scale`;
// the input columns hold lin <= L entries (zero-padded to L on load).  Complex views, FP32
// or FP64 after their dtype; `big` is the two-pass plan of L when L is longer than a tile.
fm_status exec_dft(int64_t L, const BigPlan* big, int dir, const View& in, int64_t lin, const View& out,
                   int64_t ncols, double scale, Ctx& ctx);

// Single-column FP64 DFT used at construction (spectra): out = F x (dir -1) of length L.
fm_status construction_fft64(const double2* in, double2* out, int64_t L, const BigPlan* big, cudaStream_t st);
fm_status make_big_plan(int64_t L, BigPlan* plan, cudaStream_t st);
void free_big_plan(BigPlan* plan);

}  // namespace fm
