// FP32 (complex64) instantiation of the batched FFT engine.
#include "fft_impl.cuh"
namespace fm {
template fm_status fft_launch<float>(FftArgs<float>, cudaStream_t);
template int fft_max_tile<float>();
}  // namespace fm
