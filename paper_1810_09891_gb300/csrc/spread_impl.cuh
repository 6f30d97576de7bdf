// Step B^H of Algorithm "adjoint NFFT" (Section 2): g_l = sum_{j in I^T_{n,m}(l)} f_j psi~(x_j - l/n).
//
// GPU form of the paper's blockwise adjoint (Section 3.1, Table tab:nfftflags,
// NFFT_OMP_BLOCKWISE_ADJOINT): the grid is cut into bins, and each CTA takes one subproblem
// (at most kMaxSub sorted nodes of one bin). It accumulates their contributions into a
// shared-memory tile covering the bin plus a halo of m cells on each side (shared-memory
// atomics), then adds the tile into the global grid with one vector atomic per complex cell.
// The kernel is persistent: a grid of a few CTAs per SM walks the subproblem list, whose
// length is read from device memory (it is only known on the device after the sort).
#pragma once

#include "gbnfft_internal.cuh"
#include "window.cuh"

namespace gbnfft {
namespace detail {



static __device__ __forceinline__ void global_add(float2 *p, float re, float im)
{
    atomicAdd(p, make_float2(re, im));  // vector reduction (sm_90 and later)
}
static __device__ __forceinline__ void global_add(double2 *p, double re, double im)
{
    atomicAdd(&p->x, re);
    atomicAdd(&p->y, im);
}

template <typename T, int D, int MM, int START>
__device__ __forceinline__ void spread_node(const Geom &g, T *tile, const int *tdim,
                                            const int *loc, const T *frac, T vr, T vi)
{
    constexpr int NT = 2 * MM + 1;
    if (D == 1) {
        const T b0 = (T)g.win[0].b, k0 = (T)g.win[0].kscale;
#pragma unroll
        for (int i = START; i < NT; i++) {
            const T w = psibar_tap<T>(i, MM, frac[0], b0, k0);
            T *c = tile + 2 * (loc[0] + i);
            atomicAdd(c, vr * w);
            atomicAdd(c + 1, vi * w);
        }
    } else if (D == 2) {
        T w1[NT];
        const T b1 = (T)g.win[1].b, k1 = (T)g.win[1].kscale;
#pragma unroll
        for (int i = START; i < NT; i++) w1[i] = psibar_tap<T>(i, MM, frac[1], b1, k1);
        const T b0 = (T)g.win[0].b, k0 = (T)g.win[0].kscale;
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = psibar_tap<T>(i0, MM, frac[0], b0, k0);
            const T ar = vr * w0, ai = vi * w0;
            T *row = tile + 2 * ((loc[0] + i0) * tdim[1] + loc[1]);
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                atomicAdd(row + 2 * i1, ar * w1[i1]);
                atomicAdd(row + 2 * i1 + 1, ai * w1[i1]);
            }
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
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = psibar_tap<T>(i0, MM, frac[0], b0, k0);
            const T ar = vr * w0, ai = vi * w0;
            T *plane = tile + 2 * ((loc[0] + i0) * tdim[1] * tdim[2]);
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const T br = ar * w1[i1], bi = ai * w1[i1];
                T *row = plane + 2 * ((loc[1] + i1) * tdim[2] + loc[2]);
#pragma unroll
                for (int i2 = START; i2 < NT; i2++) {
                    atomicAdd(row + 2 * i2, br * w2[i2]);
                    atomicAdd(row + 2 * i2 + 1, bi * w2[i2]);
                }
            }
        }
    }
}

template <typename T, int D, int MM>
__global__ void __launch_bounds__(256)
    spread_kernel(Geom g, const typename Cplx<T>::type *__restrict__ f,
                  const typename RecOf<T>::type *__restrict__ rec, const int *__restrict__ perm,
                  const SubProb *__restrict__ subs, const int *__restrict__ nsub_total,
                  typename Cplx<T>::type *__restrict__ grid)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    int tdim[D];
    int cells = 1;
#pragma unroll
    for (int t = 0; t < D; t++) {
        tdim[t] = g.bs[t] + 2 * MM;
        cells *= tdim[t];
    }
    const int nsub = *nsub_total;
    for (int sp = blockIdx.x; sp < nsub; sp += gridDim.x) {
        const SubProb P = subs[sp];
        int origin[D];
        {
            int b = P.bin;
#pragma unroll
            for (int t = D - 1; t >= 0; t--) {
                origin[t] = (b % g.nb[t]) * g.bs[t];
                b /= g.nb[t];
            }
        }
        for (int e = threadIdx.x; e < 2 * cells; e += blockDim.x) tile[e] = (T)0;
        __syncthreads();

        for (int k = threadIdx.x; k < P.count; k += blockDim.x) {
            const int s = P.start + k;
            const typename RecOf<T>::type r = rec[s];
            const C v = f[perm[s]];
            int cell = r.cell;
            int loc[D];
            T frac[D];
            bool edge = false;
#pragma unroll
            for (int t = D - 1; t >= 0; t--) {
                loc[t] = (cell & (g.n[t] - 1)) - origin[t];  // in [0, bs_t)
                cell >>= g.nlog[t];
                frac[t] = r.fr[t];
                edge |= (frac[t] == (T)0);
            }
            if (!edge)
                spread_node<T, D, MM, 1>(g, tile, tdim, loc, frac, v.x, v.y);
            else
                spread_node<T, D, MM, 0>(g, tile, tdim, loc, frac, v.x, v.y);
        }
        __syncthreads();

        // flush: tile cell (a_0..a_{d-1}) is grid point (origin_t - m + a_t) mod n_t
        for (int e = threadIdx.x; e < cells; e += blockDim.x) {
            const T re = tile[2 * e], im = tile[2 * e + 1];
            if (re == (T)0 && im == (T)0) continue;
            int rem = e;
            size_t gi = 0;
            int a[D];
#pragma unroll
            for (int t = D - 1; t >= 0; t--) {
                a[t] = rem % tdim[t];
                rem /= tdim[t];
            }
#pragma unroll
            for (int t = 0; t < D; t++)
                gi = (gi << g.nlog[t]) | (size_t)((origin[t] - MM + a[t]) & (g.n[t] - 1));
            global_add(grid + gi, re, im);
        }
        __syncthreads();
    }
}

template <typename T, int D, int MM>
cudaError_t launch_spread_m(const Geom &g, const typename Cplx<T>::type *f,
                            const typename RecOf<T>::type *rec, const int *perm,
                            const SubProb *subs, const int *nsub_total, int max_subs,
                            typename Cplx<T>::type *grid, cudaStream_t stream)
{
    size_t cells = 1;
    for (int t = 0; t < D; t++) cells *= (size_t)(g.bs[t] + 2 * MM);
    const size_t smem = cells * 2 * sizeof(T);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(spread_kernel<T, D, MM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = 256;
    int per_sm = (int)((200 * 1024) / (smem + 1024));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    int blocks = num_sms() * per_sm;
    if (blocks > max_subs) blocks = max_subs;
    if (blocks < 1) blocks = 1;
    spread_kernel<T, D, MM><<<blocks, threads, smem, stream>>>(g, f, rec, perm, subs, nsub_total,
                                                               grid);
    return cudaGetLastError();
}



template <typename T, int D>
cudaError_t spread_d(const Geom &g, const typename Cplx<T>::type *f,
                     const typename RecOf<T>::type *rec, const int *perm, const SubProb *subs,
                     const int *nsub_total, int max_subs, typename Cplx<T>::type *grid,
                     cudaStream_t stream)
{
    GBNFFT_DISPATCH_M(launch_spread_m, T, D, g, f, rec, perm, subs, nsub_total, max_subs, grid,
                      stream)
}

}  // namespace detail
}  // namespace gbnfft
