// Instantiation unit: grad kernels, float, d = 1, window cutoffs m = 1..kMaxM.
#include "interp_impl.cuh"

namespace gbnfft {
namespace detail {
template cudaError_t grad_d<float, 1>(const Geom &, const float2 *, const RecF *, const int *, int64_t, const float2 *, float *, cudaStream_t);
}  // namespace detail
}  // namespace gbnfft
