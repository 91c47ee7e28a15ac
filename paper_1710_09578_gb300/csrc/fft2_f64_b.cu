// Instantiations of the compile-time-length FFT tile kernel: double, log2 L in [9, 13].
#include "fft2.cuh"

namespace fm {

fm_status fft2_dispatch_f64_b(const FftArgs<double>& a, int logL, cudaStream_t st) {
  switch (logL) {
    case 9: return fft2_launch<double, 9>(a, st);
    case 10: return fft2_launch<double, 10>(a, st);
    case 11: return fft2_launch<double, 11>(a, st);
    case 12: return fft2_launch<double, 12>(a, st);
    case 13: return fft2_launch<double, 13>(a, st);
    default: break;
  }
  set_error("fft: no kernel for log2 L = %d", logL);
  return FM_ERR_UNSUPPORTED;
}

}  // namespace fm
