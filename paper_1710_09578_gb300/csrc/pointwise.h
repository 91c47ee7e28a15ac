// Launchers of the pointwise / setup kernels (pointwise.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fm_internal.h"

namespace fm {

// Output element (c, o, t, i) of a view [ncols][outer][n_out][inner] reads input element
// (c, o, map[t] or t, i) (zero if map[t] < 0), multiplies by d[src] (conj if d_conj) and
// scale, and stores (or accumulates when beta = 1).
struct PwArgs {
  int64_t ncols = 0, outer = 1, inner = 1, n_out = 0;
  const void* in = nullptr;
  int64_t in_ld = 0, in_ostride = 0;
  int in_cplx = 0;
  void* out = nullptr;
  int64_t out_ld = 0, out_ostride = 0;
  int out_cplx = 0;
  const int32_t* map = nullptr;
  const void* dc = nullptr;   // complex diagonal (float2 / double2)
  const void* dr = nullptr;   // real diagonal (float / double)
  int d_conj = 0;
  double scale = 1.0;
  int beta = 0;
};

fm_status pointwise_launch(const PwArgs& a, bool dbl, cudaStream_t st);
fm_status i32_copy_launch(const int* in, int64_t in_ld, int* out, int64_t out_ld, int64_t n, int64_t ncols,
                          int beta, cudaStream_t st);
fm_status twiddle_launch(int64_t N, float2* t32, double2* t64, cudaStream_t st);
// the pass-twiddle tables of the Stockham passes (layout: pass_tw_offset in fm_device.cuh)
fm_status pass_twiddle_launch(float2* t32, double2* t64, cudaStream_t st);
fm_status spectrum_finish_launch(double2* s64, float2* s32, double2* p64, float2* p32, int64_t L, int64_t N1,
                                 int64_t N2, double scale, cudaStream_t st);
fm_status to_c128_launch(const void* src, fm_dtype dt, int64_t n, int64_t dst_len, double2* dst, cudaStream_t st);
fm_status toeplitz_embed_launch(const double2* t, int64_t rows, int64_t cols, int64_t L, double2* c,
                                cudaStream_t st);
fm_status diag_finish_launch(const double2* d, int64_t n, float2* d32, double* dr64, float* dr32, cudaStream_t st);
fm_status spec_cap_launch(const double2* s, int64_t L, double scale, double* out, cudaStream_t st);

}  // namespace fm
