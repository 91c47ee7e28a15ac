// Instantiations of the compile-time-length FFT tile kernel: float, log2 L in [12, 14].
#include "fft2.cuh"

namespace fm {

fm_status fft2_dispatch_f32_c(const FftArgs<float>& a, int logL, cudaStream_t st) {
  switch (logL) {
    case 12: return fft2_launch<float, 12>(a, st);
    case 13: return fft2_launch<float, 13>(a, st);
    case 14: return fft2_launch<float, 14>(a, st);
    default: break;
  }
  set_error("fft: no kernel for log2 L = %d", logL);
  return FM_ERR_UNSUPPORTED;
}

}  // namespace fm
