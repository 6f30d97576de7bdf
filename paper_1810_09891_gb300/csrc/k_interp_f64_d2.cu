// Instantiation unit: interp kernels, double, d = 2, window cutoffs m = 1..kMaxM.
#include "interp_impl.cuh"

namespace gbnfft {
namespace detail {
template cudaError_t interp_d<double, 2>(const Geom &, const double2 *, const RecD *, const int *, int64_t, const SubProb *, const int *, int, double2 *, cudaStream_t);
}  // namespace detail
}  // namespace gbnfft
