// Launch descriptor of the batched FFT tile kernel (fft2.cuh).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {

enum IoMode { IO_C = 0, IO_R = 1, IO_RP = 2 };

// Vectors are g = (c, o, i) with i fastest: c in [0, ncu) column units (columns, or pairs
// of real columns in IO_RP mode), o in [0, outer), i in [0, inner).  On each side X (in,
// out) element t of vector g is
//   X[c*X_ld + o*X_ostride + (i % X_imod) + src*X_tstride],
//   n   = t*X_fmul + ((o*inner + i) / X_fdiv) % X_fmod      (position in the operator's axis)
//   src = n, or pre_map[n] / post_map[n] when a row selection is fused.
// Plain views use X_fmul = 1, X_fmod = 1 (n = t) and X_imod = inner.  The passes of the
// two-pass plan for long transforms use the other settings to address the original axis.
template <typename T>
struct FftArgs {
  typedef typename Cx<T>::t C;
  // transform
  int64_t L = 0;
  int logL = 0;
  int dir0 = -1;            // -1 forward (exp(-i...)), +1 inverse, for the first transform
  int conv = 0;             // 1: transform, x spectrum, inverse transform
  const C* spec = nullptr;  // length L (times spec_omod rows for per-row spectra)
  int64_t spec_omod = 1;    // spectrum row = o % spec_omod
  int spec_conj = 0;
  const C* tw = nullptr;    // pass-twiddle tables (pass_tw_offset)
  // geometry
  int64_t ncu = 0, ncols = 0, outer = 1, inner = 1;
  int V = 1, logV = 0;
  int small = 0;            // 1: small tiles (passes of a small two-pass FP64 problem)
  int tile = 0;             // tile shape of strided views: 0 automatic, 1 default, 2 wide, 3 wide in 4 groups
  int rcap = 0;             // 3: radices of at most 8 (compiled for FP32 tiles of 2^9 .. 2^12)
  int out_stage = 0;        // 1: outputs transposed through shared memory (set by the launcher)
  // input view
  const void* in = nullptr;
  int64_t in_ld = 0, in_ostride = 0, in_tstride = 1;
  int64_t in_fmul = 1, in_fdiv = 1, in_fmod = 1, in_imod = 1;
  int in_mode = IO_C;
  int64_t Lin = 0;
  int in_vcontig = 0;
  // output view
  void* out = nullptr;
  int64_t out_ld = 0, out_ostride = 0, out_tstride = 1;
  int64_t out_fmul = 1, out_fdiv = 1, out_fmod = 1, out_imod = 1;
  int out_mode = IO_C;
  int64_t Lout = 0;
  int out_vcontig = 0;
  // twiddle index t * ((o*inner + i) / tw_div % tw_mod) of the two-pass plan
  int64_t tw_div = 1, tw_mod = 1;
  // pre ops (on load)
  const int32_t* pre_map = nullptr;
  const C* pre_dc = nullptr;
  const T* pre_dr = nullptr;
  int pre_conj = 0;
  const C* pre_tw = nullptr;
  int64_t tw_mask = 0;
  int pre_tw_conj = 0;
  // post ops (on store)
  const C* post_tw = nullptr;
  int post_tw_conj = 0;
  const C* post_dc = nullptr;
  const T* post_dr = nullptr;
  int post_conj = 0;
  const int32_t* post_map = nullptr;
  T scale = 1;
  int beta = 0;
};

template <typename T>
fm_status fft_launch(FftArgs<T> a, cudaStream_t st);
template <typename T>
int fft_max_tile();

}  // namespace fm
