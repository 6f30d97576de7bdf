// Instantiation unit: interp kernels, float, d = 3, window cutoffs m = 1..kMaxM.
#include "interp_impl.cuh"

namespace gbnfft {
namespace detail {
template cudaError_t interp_d<float, 3>(const Geom &, const float2 *, const RecF *, const int *, int64_t, const SubProb *, const int *, int, float2 *, cudaStream_t);
}  // namespace detail
}  // namespace gbnfft
