// Instantiations of the compile-time-length FFT tile kernel: float, log2 L in [1, 7].
#include "fft2.cuh"

namespace fm {

fm_status fft2_dispatch_f32_a(const FftArgs<float>& a, int logL, cudaStream_t st) {
  switch (logL) {
    case 1: return fft2_launch<float, 1>(a, st);
    case 2: return fft2_launch<float, 2>(a, st);
    case 3: return fft2_launch<float, 3>(a, st);
    case 4: return fft2_launch<float, 4>(a, st);
    case 5: return fft2_launch<float, 5>(a, st);
    case 6: return fft2_launch<float, 6>(a, st);
    case 7: return fft2_launch<float, 7>(a, st);
    default: break;
  }
  set_error("fft: no kernel for log2 L = %d", logL);
  return FM_ERR_UNSUPPORTED;
}

}  // namespace fm
