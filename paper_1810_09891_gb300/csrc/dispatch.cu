// Dispatch of the node kernels on the dimension d (the per-d launchers live in k_*.cu).
#include "gbnfft_internal.cuh"

namespace gbnfft {

template <typename T>
cudaError_t launch_interp(const Geom &g, const typename Cplx<T>::type *grid,
                          const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                          const SubProb *subs, const int *nsub_total, int max_subs,
                          typename Cplx<T>::type *f, cudaStream_t stream)
{
    if (M == 0) return cudaSuccess;
    switch (g.d) {
    case 1: return detail::interp_d<T, 1>(g, grid, rec, perm, M, subs, nsub_total, max_subs, f, stream);
    case 2: return detail::interp_d<T, 2>(g, grid, rec, perm, M, subs, nsub_total, max_subs, f, stream);
    case 3: return detail::interp_d<T, 3>(g, grid, rec, perm, M, subs, nsub_total, max_subs, f, stream);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_grad(const Geom &g, const typename Cplx<T>::type *grid,
                        const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                        const typename Cplx<T>::type *w, T *gx, cudaStream_t stream)
{
    if (M == 0) return cudaSuccess;
    switch (g.d) {
    case 1: return detail::grad_d<T, 1>(g, grid, rec, perm, M, w, gx, stream);
    case 2: return detail::grad_d<T, 2>(g, grid, rec, perm, M, w, gx, stream);
    case 3: return detail::grad_d<T, 3>(g, grid, rec, perm, M, w, gx, stream);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_spread(const Geom &g, const typename Cplx<T>::type *f,
                          const typename RecOf<T>::type *rec, const int *perm,
                          const SubProb *subs, int *nsub_total, int max_subs,
                          typename Cplx<T>::type *grid, cudaStream_t stream)
{
    switch (g.d) {
    case 1: return detail::spread_d<T, 1>(g, f, rec, perm, subs, nsub_total, max_subs, grid, stream);
    case 2: return detail::spread_d<T, 2>(g, f, rec, perm, subs, nsub_total, max_subs, grid, stream);
    case 3: return detail::spread_d<T, 3>(g, f, rec, perm, subs, nsub_total, max_subs, grid, stream);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_interp<float>(const Geom &, const float2 *, const RecF *, const int *,
                                          int64_t, const SubProb *, const int *, int, float2 *,
                                          cudaStream_t);
template cudaError_t launch_interp<double>(const Geom &, const double2 *, const RecD *,
                                           const int *, int64_t, const SubProb *, const int *,
                                           int, double2 *, cudaStream_t);
template cudaError_t launch_grad<float>(const Geom &, const float2 *, const RecF *, const int *,
                                        int64_t, const float2 *, float *, cudaStream_t);
template cudaError_t launch_grad<double>(const Geom &, const double2 *, const RecD *, const int *,
                                         int64_t, const double2 *, double *, cudaStream_t);
template cudaError_t launch_spread<float>(const Geom &, const float2 *, const RecF *, const int *,
                                          const SubProb *, int *, int, float2 *,
                                          cudaStream_t);
template cudaError_t launch_spread<double>(const Geom &, const double2 *, const RecD *,
                                           const int *, const SubProb *, int *, int,
                                           double2 *, cudaStream_t);

}  // namespace gbnfft
