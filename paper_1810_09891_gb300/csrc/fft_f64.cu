// Instantiation unit: FFT axis passes, double.
#include "fft_impl.cuh"

namespace gbnfft {
template cudaError_t launch_fft_axis<double>(const double2 *, double2 *, int64_t, int64_t, int, int, int, int,
                                         const double2 *, const double *, cudaStream_t);
template cudaError_t launch_fft_axis_bluestein<double>(const double2 *, double2 *, int64_t, int64_t, int,
                                                   int, int, int, const double *,
                                                   const BluesteinAxis<double> &, cudaStream_t);
template cudaError_t launch_fft_fused<double>(const FusedFftPass *, const FusedItem *, int, int,
                                           size_t, const FusedPtrs &, cudaStream_t);
}  // namespace gbnfft
