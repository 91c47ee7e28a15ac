// Instantiations of the compile-time-length FFT tile kernel: double, log2 L in [1, 8].
#include "fft2.cuh"

namespace fm {

fm_status fft2_dispatch_f64_a(const FftArgs<double>& a, int logL, cudaStream_t st) {
  switch (logL) {
    case 1: return fft2_launch<double, 1>(a, st);
    case 2: return fft2_launch<double, 2>(a, st);
    case 3: return fft2_launch<double, 3>(a, st);
    case 4: return fft2_launch<double, 4>(a, st);
    case 5: return fft2_launch<double, 5>(a, st);
    case 6: return fft2_launch<double, 6>(a, st);
    case 7: return fft2_launch<double, 7>(a, st);
    case 8: return fft2_launch<double, 8>(a, st);
    default: break;
  }
  set_error("fft: no kernel for log2 L = %d", logL);
  return FM_ERR_UNSUPPORTED;
}

}  // namespace fm
