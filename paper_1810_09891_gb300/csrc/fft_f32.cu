// Instantiation unit: FFT axis passes, float.
#include "fft_impl.cuh"

namespace gbnfft {
template cudaError_t launch_fft_axis<float>(const float2 *, float2 *, int64_t, int64_t, int, int, int, int,
                                         const float2 *, const float *, cudaStream_t);
template cudaError_t launch_fft_axis_bluestein<float>(const float2 *, float2 *, int64_t, int64_t, int,
                                                   int, int, int, const float *,
                                                   const BluesteinAxis<float> &, cudaStream_t);
template cudaError_t launch_fft_fused<float>(const FusedFftPass *, const FusedItem *, int, int,
                                           size_t, const FusedPtrs &, cudaStream_t);
}  // namespace gbnfft
