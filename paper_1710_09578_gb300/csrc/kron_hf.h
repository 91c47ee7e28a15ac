// Fused outer-Hadamard / inner-Fourier mode products of a Kron operator (kron_hf.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fm_internal.h"

namespace fm {

struct KronHFArgs {
  const float2* in = nullptr;
  float2* out = nullptr;
  int64_t in_ld = 0, out_ld = 0;  // column strides (elements)
  int64_t nmid = 1;               // product of the lengths of the middle axes
  int64_t ntiles = 0;             // columns x nmid
  int64_t sa = 0;                 // stride of the Hadamard (outermost) axis: nmid * 2^LB
  int dir = -1;                   // Fourier direction: -1 forward, +1 adjoint
  float scale = 1.f;              // 1, or 1/sqrt(2^LB) for the orthonormal Fourier matrix
  int beta = 0;                   // 1: accumulate into out
  const float2* tw = nullptr;     // pass-twiddle tables (pass_tw_offset)
  int pair = 0;                   // each tile on one CTA (0), a cluster of 2 (1) or of 4 CTAs (2), or
                                  // of 2 CTAs that prefetch a later tile's rows into L2 (3)
  int64_t pf_tiles = 0;           // > 0: prefetch into L2 the rows of tile + pf_tiles (set by the launcher)
};

// Tiles [2^la][2^lb] with 2^10 <= 2^(la+lb) <= 2^14 and 4 <= la, lb <= 8.
bool kron_hf_ok(int la, int lb);
fm_status kron_hf_launch(const KronHFArgs& a, int la, int lb, cudaStream_t st);

}  // namespace fm
