// Instantiations of the compile-time-length FFT tile kernel: float, log2 L in [8, 11].
#include "fft2.cuh"

namespace fm {

fm_status fft2_dispatch_f32_b(const FftArgs<float>& a, int logL, cudaStream_t st) {
  switch (logL) {
    case 8: return fft2_launch<float, 8>(a, st);
    case 9: return fft2_launch<float, 9>(a, st);
    case 10: return fft2_launch<float, 10>(a, st);
    case 11: return fft2_launch<float, 11>(a, st);
    default: break;
  }
  set_error("fft: no kernel for log2 L = %d", logL);
  return FM_ERR_UNSUPPORTED;
}

}  // namespace fm
