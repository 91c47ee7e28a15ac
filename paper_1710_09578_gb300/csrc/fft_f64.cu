// FP64 (complex128) instantiation of the batched FFT engine.
#include "fft_impl.cuh"
namespace fm {
template fm_status fft_launch<double>(FftArgs<double>, cudaStream_t);
template int fft_max_tile<double>();
}  // namespace fm
