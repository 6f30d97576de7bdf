// Instantiation unit: FFT axis passes, float.
#include "fft_impl.cuh"

namespace gbnfft {
template cudaError_t launch_fft_axis<float>(const float2 *, float2 *, int64_t, int64_t, int, int, bool, int,
                                         const float2 *, const float *, cudaStream_t);
}  // namespace gbnfft
