// Instantiation unit: spread kernels, float, d = 3, window cutoffs m = 1..kMaxM.
#include "spread_impl.cuh"

namespace gbnfft {
namespace detail {
template cudaError_t spread_d<float, 3>(const Geom &, const float2 *, const RecF *, const int *, const SubProb *, int *, int, float2 *, cudaStream_t);
}  // namespace detail
}  // namespace gbnfft
