// Launch descriptors of the Walsh-Hadamard kernels (fwht.cu, fwht_mma.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fm_internal.h"

namespace fm {

// Vectors g = (c, o, i), i fastest; element t of vector g at c*ld + o*ostride + t*tstride + i.
struct FwhtArgs {
  int logL = 0;                        // transform length 2^logL
  int logLp = 0, logC = 0, logV = 0;   // set by the launcher
  int64_t ncols = 0, outer = 1, inner = 1;
  const void* in = nullptr;
  int64_t in_ld = 0, in_ostride = 0, in_tstride = 1;
  void* out = nullptr;
  int64_t out_ld = 0, out_ostride = 0, out_tstride = 1;
  int beta = 0;
  int prefetch = 1;  // long contiguous columns: 1 prefetch a later column's blocks into L2, 0 not
};

fm_status fwht_launch(FwhtArgs a, fm_dtype in_dt, cudaStream_t st);
// Strided axes (inner >= 16), n <= 256: compile-time-length kernel (fwht2.cu).
bool fwht2_ok(const FwhtArgs& a);
fm_status fwht2_launch(const FwhtArgs& a, fm_dtype in_dt, cudaStream_t st);
// BF16 tensor-core variants: split = 0 plain BF16 operands, 1 hi + lo split.
fm_status fwht_mma_launch(FwhtArgs a, int split, cudaStream_t st);

}  // namespace fm
