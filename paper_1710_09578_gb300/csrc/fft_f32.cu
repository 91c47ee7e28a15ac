// FP32 (complex64) entry of the batched FFT engine: dispatch on the transform length.
#include "fft_impl.cuh"

namespace fm {

fm_status fft2_dispatch_f32_a(const FftArgs<float>& a, int logL, cudaStream_t st);
fm_status fft2_dispatch_f32_b(const FftArgs<float>& a, int logL, cudaStream_t st);
fm_status fft2_dispatch_f32_c(const FftArgs<float>& a, int logL, cudaStream_t st);

template <>
fm_status fft_launch<float>(FftArgs<float> a, cudaStream_t st) {
  if (a.L < 2 || (a.L & (a.L - 1)) || a.L > fft_max_tile<float>()) {
    set_error("fft: unsupported single-tile length %lld", (long long)a.L);
    return FM_ERR_UNSUPPORTED;
  }
  int logL = 0;
  while ((1LL << logL) < a.L) ++logL;
  if (logL < 8) return fft2_dispatch_f32_a(a, logL, st);
  if (logL < 12) return fft2_dispatch_f32_b(a, logL, st);
  return fft2_dispatch_f32_c(a, logL, st);
}

template int fft_max_tile<float>();

}  // namespace fm
