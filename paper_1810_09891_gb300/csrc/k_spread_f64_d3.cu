// Instantiation unit: spread kernels, double, d = 3, window cutoffs m = 1..kMaxM.
#include "spread_impl.cuh"

namespace gbnfft {
namespace detail {
template cudaError_t spread_d<double, 3>(const Geom &, const double2 *, const RecD *, const int *, const SubProb *, int *, int, double2 *, cudaStream_t);
}  // namespace detail
}  // namespace gbnfft
