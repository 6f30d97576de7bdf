// Step B of Algorithm "NFFT" (Section 2, eq. s_approx): for every node,
//   f_j = sum_{l in I_{n,m}(x_j)} g_{l mod n} prod_t psi_t(n_t x_{j,t} - l_t),
// and the derivative of the same sum with respect to the node coordinates (node gradient).
//
// One thread per node, nodes visited in bin-sorted order so that the threads of a warp read
// neighbouring grid cells (L1/L2 reuse of the oversampled grid). The window weights of the
// inner axes are computed once per node into registers; the outermost axis weight is computed
// in the outer loop. Nodes whose offset on some axis is exactly 0 (a node on a grid point) use
// 2m+1 taps per axis; all other nodes use 2m (the closed support of eq. Inm).
#pragma once

#include "gbnfft_internal.cuh"
#include "window.cuh"

namespace gbnfft {
namespace detail {



template <typename T, int D, int MM, int START>
__device__ __forceinline__ typename Cplx<T>::type
interp_node(const Geom &g, const typename Cplx<T>::type *__restrict__ grid, const int *base,
            const T *frac)
{
    using C = typename Cplx<T>::type;
    constexpr int NT = 2 * MM + 1;
    C acc;
    acc.x = (T)0;
    acc.y = (T)0;
    if (D == 1) {
        const T b0 = (T)g.win[0].b, k0 = (T)g.win[0].kscale;
        const int mask0 = g.n[0] - 1;
#pragma unroll
        for (int i = START; i < NT; i++) {
            const T w = psibar_tap<T>(i, MM, frac[0], b0, k0);
            const C v = grid[(base[0] - MM + i) & mask0];
            acc.x += v.x * w;
            acc.y += v.y * w;
        }
    } else if (D == 2) {
        T w1[NT];
        const T b1 = (T)g.win[1].b, k1 = (T)g.win[1].kscale;
#pragma unroll
        for (int i = START; i < NT; i++) w1[i] = psibar_tap<T>(i, MM, frac[1], b1, k1);
        const T b0 = (T)g.win[0].b, k0 = (T)g.win[0].kscale;
        const int mask0 = g.n[0] - 1, mask1 = g.n[1] - 1, sh0 = g.nlog[1];
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = psibar_tap<T>(i0, MM, frac[0], b0, k0);
            const C *row = grid + ((size_t)((base[0] - MM + i0) & mask0) << sh0);
            C in;
            in.x = (T)0;
            in.y = (T)0;
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const C v = row[(base[1] - MM + i1) & mask1];
                in.x += v.x * w1[i1];
                in.y += v.y * w1[i1];
            }
            acc.x += in.x * w0;
            acc.y += in.y * w0;
        }
    } else {
        T w1[NT], w2[NT];
        const T b1 = (T)g.win[1].b, k1 = (T)g.win[1].kscale;
        const T b2 = (T)g.win[2].b, k2 = (T)g.win[2].kscale;
#pragma unroll
        for (int i = START; i < NT; i++) {
            w1[i] = psibar_tap<T>(i, MM, frac[1], b1, k1);
            w2[i] = psibar_tap<T>(i, MM, frac[2], b2, k2);
        }
        const T b0 = (T)g.win[0].b, k0 = (T)g.win[0].kscale;
        const int mask0 = g.n[0] - 1, mask1 = g.n[1] - 1, mask2 = g.n[2] - 1;
        const int sh1 = g.nlog[2], sh0 = g.nlog[1] + g.nlog[2];
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = psibar_tap<T>(i0, MM, frac[0], b0, k0);
            const C *plane = grid + ((size_t)((base[0] - MM + i0) & mask0) << sh0);
            C pl;
            pl.x = (T)0;
            pl.y = (T)0;
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const C *row = plane + ((size_t)((base[1] - MM + i1) & mask1) << sh1);
                C in;
                in.x = (T)0;
                in.y = (T)0;
#pragma unroll
                for (int i2 = START; i2 < NT; i2++) {
                    const C v = row[(base[2] - MM + i2) & mask2];
                    in.x += v.x * w2[i2];
                    in.y += v.y * w2[i2];
                }
                pl.x += in.x * w1[i1];
                pl.y += in.y * w1[i1];
            }
            acc.x += pl.x * w0;
            acc.y += pl.y * w0;
        }
    }
    return acc;
}

template <typename T, int D>
__device__ __forceinline__ void decode_node(const Geom &g, const typename RecOf<T>::type &r,
                                            int *base, T *frac, bool &edge)
{
    int cell = r.cell;
    edge = false;
#pragma unroll
    for (int t = D - 1; t >= 0; t--) {
        base[t] = cell & (g.n[t] - 1);
        cell >>= g.nlog[t];
        frac[t] = r.fr[t];
        edge |= (frac[t] == (T)0);
    }
}

template <typename T, int D, int MM>
__global__ void __launch_bounds__(128)
    interp_kernel(Geom g, const typename Cplx<T>::type *__restrict__ grid,
                  const typename RecOf<T>::type *__restrict__ rec, const int *__restrict__ perm,
                  int M, typename Cplx<T>::type *__restrict__ f)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const typename RecOf<T>::type r = rec[s];
    int base[D];
    T frac[D];
    bool edge;
    decode_node<T, D>(g, r, base, frac, edge);
    typename Cplx<T>::type v;
    if (!edge)
        v = interp_node<T, D, MM, 1>(g, grid, base, frac);
    else
        v = interp_node<T, D, MM, 0>(g, grid, base, frac);
    f[perm[s]] = v;
}

// Node gradient: accumulates, per axis t, sum_l g_l dpsibar_t(.) prod_{u != t} psibar_u(.).
template <typename T, int D, int MM, int START>
__device__ __forceinline__ void grad_node(const Geom &g,
                                          const typename Cplx<T>::type *__restrict__ grid,
                                          const int *base, const T *frac,
                                          typename Cplx<T>::type *acc)
{
    using C = typename Cplx<T>::type;
    constexpr int NT = 2 * MM + 1;
#pragma unroll
    for (int t = 0; t < D; t++) {
        acc[t].x = (T)0;
        acc[t].y = (T)0;
    }
    if (D == 1) {
        const T b0 = (T)g.win[0].b, k0 = (T)g.win[0].kscale;
        const int mask0 = g.n[0] - 1;
#pragma unroll
        for (int i = START; i < NT; i++) {
            const T dw = dpsibar_tap<T>(i, MM, frac[0], b0, k0);
            const C v = grid[(base[0] - MM + i) & mask0];
            acc[0].x += v.x * dw;
            acc[0].y += v.y * dw;
        }
    } else if (D == 2) {
        T w1[NT], d1[NT];
        const T b1 = (T)g.win[1].b, k1 = (T)g.win[1].kscale;
#pragma unroll
        for (int i = START; i < NT; i++) {
            w1[i] = psibar_tap<T>(i, MM, frac[1], b1, k1);
            d1[i] = dpsibar_tap<T>(i, MM, frac[1], b1, k1);
        }
        const T b0 = (T)g.win[0].b, k0 = (T)g.win[0].kscale;
        const int mask0 = g.n[0] - 1, mask1 = g.n[1] - 1, sh0 = g.nlog[1];
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = psibar_tap<T>(i0, MM, frac[0], b0, k0);
            const T d0 = dpsibar_tap<T>(i0, MM, frac[0], b0, k0);
            const C *row = grid + ((size_t)((base[0] - MM + i0) & mask0) << sh0);
            C s0, s1;
            s0.x = s0.y = s1.x = s1.y = (T)0;
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const C v = row[(base[1] - MM + i1) & mask1];
                s0.x += v.x * w1[i1];
                s0.y += v.y * w1[i1];
                s1.x += v.x * d1[i1];
                s1.y += v.y * d1[i1];
            }
            acc[0].x += s0.x * d0;
            acc[0].y += s0.y * d0;
            acc[1].x += s1.x * w0;
            acc[1].y += s1.y * w0;
        }
    } else {
        T w1[NT], d1[NT], w2[NT], d2[NT];
        const T b1 = (T)g.win[1].b, k1 = (T)g.win[1].kscale;
        const T b2 = (T)g.win[2].b, k2 = (T)g.win[2].kscale;
#pragma unroll
        for (int i = START; i < NT; i++) {
            w1[i] = psibar_tap<T>(i, MM, frac[1], b1, k1);
            d1[i] = dpsibar_tap<T>(i, MM, frac[1], b1, k1);
            w2[i] = psibar_tap<T>(i, MM, frac[2], b2, k2);
            d2[i] = dpsibar_tap<T>(i, MM, frac[2], b2, k2);
        }
        const T b0 = (T)g.win[0].b, k0 = (T)g.win[0].kscale;
        const int mask0 = g.n[0] - 1, mask1 = g.n[1] - 1, mask2 = g.n[2] - 1;
        const int sh1 = g.nlog[2], sh0 = g.nlog[1] + g.nlog[2];
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = psibar_tap<T>(i0, MM, frac[0], b0, k0);
            const T d0 = dpsibar_tap<T>(i0, MM, frac[0], b0, k0);
            const C *plane = grid + ((size_t)((base[0] - MM + i0) & mask0) << sh0);
            C p0, p1, p2;  // plane sums for the three partial derivatives
            p0.x = p0.y = p1.x = p1.y = p2.x = p2.y = (T)0;
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const C *row = plane + ((size_t)((base[1] - MM + i1) & mask1) << sh1);
                C sw, sd;
                sw.x = sw.y = sd.x = sd.y = (T)0;
#pragma unroll
                for (int i2 = START; i2 < NT; i2++) {
                    const C v = row[(base[2] - MM + i2) & mask2];
                    sw.x += v.x * w2[i2];
                    sw.y += v.y * w2[i2];
                    sd.x += v.x * d2[i2];
                    sd.y += v.y * d2[i2];
                }
                p0.x += sw.x * w1[i1];  // -> d0 * w1 * w2
                p0.y += sw.y * w1[i1];
                p1.x += sw.x * d1[i1];  // -> w0 * d1 * w2
                p1.y += sw.y * d1[i1];
                p2.x += sd.x * w1[i1];  // -> w0 * w1 * d2
                p2.y += sd.y * w1[i1];
            }
            acc[0].x += p0.x * d0;
            acc[0].y += p0.y * d0;
            acc[1].x += p1.x * w0;
            acc[1].y += p1.y * w0;
            acc[2].x += p2.x * w0;
            acc[2].y += p2.y * w0;
        }
    }
}

template <typename T, int D, int MM>
__global__ void __launch_bounds__(128)
    grad_kernel(Geom g, const typename Cplx<T>::type *__restrict__ grid,
                const typename RecOf<T>::type *__restrict__ rec, const int *__restrict__ perm,
                int M, const typename Cplx<T>::type *__restrict__ w, T *__restrict__ gx)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const typename RecOf<T>::type r = rec[s];
    int base[D];
    T frac[D];
    bool edge;
    decode_node<T, D>(g, r, base, frac, edge);
    typename Cplx<T>::type acc[D];
    if (!edge)
        grad_node<T, D, MM, 1>(g, grid, base, frac, acc);
    else
        grad_node<T, D, MM, 0>(g, grid, base, frac, acc);
    const int j = perm[s];
    const typename Cplx<T>::type wj = w[j];
#pragma unroll
    for (int t = 0; t < D; t++) {
        // Re(conj(w) * n_t * acc_t): the chain rule d/dx_t = n_t d/d(n_t x_t)
        gx[(size_t)j * D + t] = (T)g.n[t] * (wj.x * acc[t].x + wj.y * acc[t].y);
    }
}

template <typename T, int D, int MM>
cudaError_t launch_interp_m(const Geom &g, const typename Cplx<T>::type *grid,
                            const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                            typename Cplx<T>::type *f, cudaStream_t stream)
{
    const int threads = 128;
    interp_kernel<T, D, MM><<<(unsigned)((M + threads - 1) / threads), threads, 0, stream>>>(
        g, grid, rec, perm, (int)M, f);
    return cudaGetLastError();
}

template <typename T, int D, int MM>
cudaError_t launch_grad_m(const Geom &g, const typename Cplx<T>::type *grid,
                          const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                          const typename Cplx<T>::type *w, T *gx, cudaStream_t stream)
{
    const int threads = 128;
    grad_kernel<T, D, MM><<<(unsigned)((M + threads - 1) / threads), threads, 0, stream>>>(
        g, grid, rec, perm, (int)M, w, gx);
    return cudaGetLastError();
}



template <typename T, int D>
cudaError_t interp_d(const Geom &g, const typename Cplx<T>::type *grid,
                     const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                     typename Cplx<T>::type *f, cudaStream_t stream)
{
    GBNFFT_DISPATCH_M(launch_interp_m, T, D, g, grid, rec, perm, M, f, stream)
}

template <typename T, int D>
cudaError_t grad_d(const Geom &g, const typename Cplx<T>::type *grid,
                   const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                   const typename Cplx<T>::type *w, T *gx, cudaStream_t stream)
{
    GBNFFT_DISPATCH_M(launch_grad_m, T, D, g, grid, rec, perm, M, w, gx, stream)
}

}  // namespace detail
}  // namespace gbnfft
