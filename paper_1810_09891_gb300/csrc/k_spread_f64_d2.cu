// Instantiation unit: spread kernels, double, d = 2, window cutoffs m = 1..kMaxM.
#include "spread_impl.cuh"

namespace gbnfft {
namespace detail {
template cudaError_t spread_d<double, 2>(const Geom &, const double2 *, const RecD *, const int *, const SubProb *, int *, int, double2 *, cudaStream_t);
}  // namespace detail
}  // namespace gbnfft
