// FP64 (complex128) entry of the batched FFT engine: dispatch on the transform length.
#include "fft_impl.cuh"

namespace fm {

fm_status fft2_dispatch_f64_a(const FftArgs<double>& a, int logL, cudaStream_t st);
fm_status fft2_dispatch_f64_b(const FftArgs<double>& a, int logL, cudaStream_t st);

template <>
fm_status fft_launch<double>(FftArgs<double> a, cudaStream_t st) {
  if (a.L < 2 || (a.L & (a.L - 1)) || a.L > fft_max_tile<double>()) {
    set_error("fft: unsupported single-tile length %lld", (long long)a.L);
    return FM_ERR_UNSUPPORTED;
  }
  int logL = 0;
  while ((1LL << logL) < a.L) ++logL;
  if (logL < 9) return fft2_dispatch_f64_a(a, logL, st);
  return fft2_dispatch_f64_b(a, logL, st);
}

template int fft_max_tile<double>();

}  // namespace fm
