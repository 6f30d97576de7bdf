// Step B of Algorithm "NFFT" (Section 2, eq. s_approx): for every node,
//   f_j = sum_{l in I_{n,m}(x_j)} g_{l mod n} prod_t psi_t(n_t x_{j,t} - l_t),
// and the derivative of the same sum with respect to the node coordinates (node gradient).
//
// Thread form (default): one thread per node, nodes visited in bin-sorted
// order so that the threads of a warp read neighbouring grid cells (L1/L2 reuse of the
// oversampled grid). The window values of the inner axes are evaluated once per node into
// registers from the per-tap polynomials (kernel-argument tables, read as warp-wide
// broadcasts); the outermost axis' value is evaluated in the outer loop. Nodes whose offset on some axis is exactly 0 (a
// node on a grid point) use 2m+1 taps per axis; all other nodes use 2m (the closed support of
// eq. Inm).
//
// Warp form (option): one warp per node, the lanes cover the node's taps. Octet form (option,
// d = 2, 3 with m <= 4): eight lanes per node along the last axis (see below). Tiled form
// (option): gathers from a shared-memory copy of the bin's tile.
#pragma once

#include "gbnfft_internal.cuh"
#include "window.cuh"

namespace gbnfft {
namespace detail {

constexpr int kInterpThreads = 128;

template <typename T, int D>
__device__ __forceinline__ void decode_node(const Geom &g, const typename RecOf<T>::type &r,
                                            int *base, T *frac, bool &edge)
{
    int cell = r.cell;
    edge = false;
#pragma unroll
    for (int t = D - 1; t >= 0; t--) {
        base[t] = cell & g.cmask[t];
        cell >>= g.cbits[t];
        frac[t] = r.fr[t];
        edge |= (frac[t] == (T)0);
    }
}

// FP32 rows in pairs of cells: the NC = 2m + 1 - START cells of a node's row segment, first
// cell s, are read as aligned 16-byte pairs starting at the even cell e0 = s - (s & 1) (the grid
// rows hold an even number of cells and start 16-byte aligned, and wrapping keeps pairs whole).
// That takes NC / 2 + 1 loads (the last one only when it holds a cell of the segment) instead of
// NC. wv[j] is the weight of cell e0 + j: the tap weight w[START + j - (s & 1)] inside the
// segment, 0 outside.
template <int MM, int START> struct PairRow {
    static constexpr int NC = 2 * MM + 1 - START;  // cells of the segment
    static constexpr int NP = NC / 2 + 1;          // pairs that cover it at either parity
};

template <int MM, int START>
__device__ __forceinline__ void pair_weights(const float *w, int odd, float *wv)
{
    constexpr int NC = PairRow<MM, START>::NC, NP = PairRow<MM, START>::NP;
#pragma unroll
    for (int j = 0; j < 2 * NP; j++) {
        const float we = j < NC ? w[START + j] : 0.0f;
        const float wo = (j >= 1 && j - 1 < NC) ? w[START + j - 1] : 0.0f;
        wv[j] = odd ? wo : we;
    }
}

template <int MM, int START>
__device__ __forceinline__ float2 row_dot_pairs(const float2 *__restrict__ row, int e0, int n,
                                                int odd, const float *wv)
{
    constexpr int NC = PairRow<MM, START>::NC, NP = PairRow<MM, START>::NP;
    const float4 *r4 = reinterpret_cast<const float4 *>(row);
    float2 in = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int p = 0; p < NP; p++) {
        if (p < NP - 1 || (NC & 1) || odd) {
            const float4 v = __ldg(r4 + (wrapn(e0 + 2 * p, n) >> 1));
            in.x += v.x * wv[2 * p] + v.z * wv[2 * p + 1];
            in.y += v.y * wv[2 * p] + v.w * wv[2 * p + 1];
        }
    }
    return in;
}

template <typename T, int D, int MM, int START, int MODE>
__device__ __forceinline__ typename Cplx<T>::type
interp_node(const Geom &g, const T *__restrict__ tab, const typename Cplx<T>::type *__restrict__ grid,
            const int *base, const T *frac)
{
    using C = typename Cplx<T>::type;
    constexpr int NT = 2 * MM + 1;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    constexpr bool PAIRS = sizeof(T) == 4;
    constexpr int NW = 2 * PairRow<MM, START>::NP;
    C acc;
    acc.x = (T)0;
    acc.y = (T)0;
    if (D == 1) {
        T w0[NT];
        eval_taps<T, MM, START, MODE>(g, tab, 0, frac[0], w0);
        const int n0 = g.n[0];
        if constexpr (PAIRS) {
            const int s0 = base[0] - MM + START, odd = s0 & 1;
            float wv[NW];
            pair_weights<MM, START>(w0, odd, wv);
            const float2 in = row_dot_pairs<MM, START>(grid, s0 - odd, n0, odd, wv);
            acc.x = in.x;
            acc.y = in.y;
        } else {
#pragma unroll
            for (int i = START; i < NT; i++) {
                const C v = grid[wrapn(base[0] - MM + i, n0)];
                acc.x += v.x * w0[i];
                acc.y += v.y * w0[i];
            }
        }
    } else if (D == 2) {
        T w1[NT], w0a[NT];
        eval_taps<T, MM, START, MODE>(g, tab + AS, 1, frac[1], w1);
        eval_taps<T, MM, START, MODE>(g, tab, 0, frac[0], w0a);
        const int n0 = g.n[0], n1 = g.n[1];
        const int s1 = base[1] - MM + START, odd = s1 & 1;
        float wv[NW];
        if constexpr (PAIRS) pair_weights<MM, START>(w1, odd, wv);
#pragma unroll
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = w0a[i0];
            const C *row = grid + (size_t)wrapn(base[0] - MM + i0, n0) * n1;
            C in;
            if constexpr (PAIRS) {
                in = row_dot_pairs<MM, START>(row, s1 - odd, n1, odd, wv);
            } else {
                in.x = (T)0;
                in.y = (T)0;
#pragma unroll
                for (int i1 = START; i1 < NT; i1++) {
                    const C v = row[wrapn(base[1] - MM + i1, n1)];
                    in.x += v.x * w1[i1];
                    in.y += v.y * w1[i1];
                }
            }
            acc.x += in.x * w0;
            acc.y += in.y * w0;
        }
    } else {
        T w1[NT], w2[NT];
        eval_taps<T, MM, START, MODE>(g, tab + AS, 1, frac[1], w1);
        eval_taps<T, MM, START, MODE>(g, tab + 2 * AS, 2, frac[2], w2);
        const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
        const int s2 = base[2] - MM + START, odd = s2 & 1;
        float wv[NW];
        if constexpr (PAIRS) pair_weights<MM, START>(w2, odd, wv);
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = eval_tap<T, MM, MODE>(g, tab, 0, i0, frac[0]);
            const C *plane = grid + (size_t)wrapn(base[0] - MM + i0, n0) * n1 * n2;
            C pl;
            pl.x = (T)0;
            pl.y = (T)0;
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const C *row = plane + (size_t)wrapn(base[1] - MM + i1, n1) * n2;
                C in;
                if constexpr (PAIRS) {
                    in = row_dot_pairs<MM, START>(row, s2 - odd, n2, odd, wv);
                } else {
                    in.x = (T)0;
                    in.y = (T)0;
#pragma unroll
                    for (int i2 = START; i2 < NT; i2++) {
                        const C v = row[wrapn(base[2] - MM + i2, n2)];
                        in.x += v.x * w2[i2];
                        in.y += v.y * w2[i2];
                    }
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

template <typename T, int D, int MM, bool LIN>
__global__ void __launch_bounds__(kInterpThreads)
    interp_kernel(Geom g, const __grid_constant__ WinCoef<T, MM> wc,
                  const typename Cplx<T>::type *__restrict__ grid,
                  const typename RecOf<T>::type *__restrict__ rec, const int *__restrict__ perm,
                  int M, typename Cplx<T>::type *__restrict__ f)
{
    const T *tab = wc.c;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const typename RecOf<T>::type r = rec[s];
    int base[D];
    T frac[D];
    bool edge;
    decode_node<T, D>(g, r, base, frac, edge);
    typename Cplx<T>::type v;
    constexpr int MODE = LIN ? 2 : 1;
    if (!edge)
        v = interp_node<T, D, MM, 1, MODE>(g, tab, grid, base, frac);
    else
        v = interp_node<T, D, MM, 0, MODE>(g, tab, grid, base, frac);
    f[perm[s]] = v;
}


// ------------------------------------------------------------------------- octet form of B
// Eight lanes per node, four nodes per warp (d = 2, 3; 2m <= 8). Lane l of a group reads cell
// l of every row segment of its node (the 2m cells of a row along the last axis), so one load
// instruction of the group reads a contiguous 8 x 8 (FP32) or 8 x 16 (FP64) bytes and a row
// costs two or three 32-byte sectors instead of one sector per cell pair. Lane l evaluates tap
// l + 1 of every axis; the outer-axis values reach the other lanes by shuffles, the lane's own
// last-axis value scales its partial sum, and three shuffle steps add the eight partial sums.
// A node on a grid point (2m + 1 taps on some axis) is done by the group's first lane alone.
template <typename T, int D, int MM, bool LIN>
__global__ void __launch_bounds__(kInterpThreads)
    interp_octet_kernel(Geom g, const typename Cplx<T>::type *__restrict__ grid,
                        const typename RecOf<T>::type *__restrict__ rec,
                        const int *__restrict__ perm, int M,
                        typename Cplx<T>::type *__restrict__ f)
{
    using C = typename Cplx<T>::type;
    constexpr int PT = 2 * MM;  // taps per axis of a node off the grid points
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    constexpr int DEG = PolyDeg<T, MM>::value;
    constexpr int MODE = LIN ? 2 : 1;
    static_assert(PT <= 8 && D >= 2, "octet form: d = 2, 3 and m <= 4");
    const T *poly = static_cast<const T *>(g.poly);
    const int lane = threadIdx.x & 31, l = lane & 7;
    const unsigned omask = 0xffu << (lane & 24);
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    if (s >= M) return;  // uniform in the group
    const typename RecOf<T>::type r = rec[s];
    int base[D];
    T frac[D];
    bool edge;
    decode_node<T, D>(g, r, base, frac, edge);
    if (edge) {  // uniform in the group
        if (l == 0) f[perm[s]] = interp_node<T, D, MM, 0, MODE>(g, poly, grid, base, frac);
        return;
    }
    const bool on = l < PT;
    T wl[D];  // psibar of tap l + 1 on each axis (0 for lanes past the 2m taps)
#pragma unroll
    for (int t = 0; t < D; t++) {
        if constexpr (LIN)
            wl[t] = on ? lin_tap<T, MM>(lin_axis<T, MM>(g.lin, g.lin_k, t), g.lin_k, l + 1,
                                        frac[t], (T)0)
                       : (T)0;
        else
            wl[t] = on ? poly_horner_tap<T, DEG>(poly + t * AS, l + 1, (T)2 * frac[t] - (T)1)
                       : (T)0;
    }
    const int nl = g.n[D - 1];
    const int col = on ? wrapn(base[D - 1] - MM + 1 + l, nl) : 0;
    C acc;
    acc.x = (T)0;
    acc.y = (T)0;
    if constexpr (D == 2) {
        const int n0 = g.n[0];
#pragma unroll
        for (int i0 = 0; i0 < PT; i0++) {
            const T w0 = __shfl_sync(omask, wl[0], i0, 8);
            if (on) {
                const C v = __ldg(grid + (size_t)wrapn(base[0] - MM + 1 + i0, n0) * nl + col);
                acc.x += v.x * w0;
                acc.y += v.y * w0;
            }
        }
    } else {
        const int n0 = g.n[0], n1 = g.n[1];
        T w1[PT];
        int roff[PT];
#pragma unroll
        for (int i1 = 0; i1 < PT; i1++) {
            w1[i1] = __shfl_sync(omask, wl[1], i1, 8);
            roff[i1] = wrapn(base[1] - MM + 1 + i1, n1) * nl + col;
        }
        for (int i0 = 0; i0 < PT; i0++) {
            const T w0 = __shfl_sync(omask, wl[0], i0, 8);
            const C *plane = grid + (size_t)wrapn(base[0] - MM + 1 + i0, n0) * n1 * nl;
            C pl;
            pl.x = (T)0;
            pl.y = (T)0;
#pragma unroll
            for (int i1 = 0; i1 < PT; i1++) {
                if (on) {
                    const C v = __ldg(plane + roff[i1]);
                    pl.x += v.x * w1[i1];
                    pl.y += v.y * w1[i1];
                }
            }
            acc.x += pl.x * w0;
            acc.y += pl.y * w0;
        }
    }
    acc.x *= wl[D - 1];
    acc.y *= wl[D - 1];
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(omask, acc.x, o, 8);
        acc.y += __shfl_xor_sync(omask, acc.y, o, 8);
    }
    if (l == 0) f[perm[s]] = acc;
}

// ------------------------------------------------------------------------- tiled form of B
// One CTA per subproblem (up to kMaxSub sorted nodes of one bin, the list built by set_nodes):
// the bin's grid tile plus a halo of m cells per side is staged in shared memory with
// row-coalesced loads, then every thread interpolates its nodes from the tile. Gathers from
// shared memory replace the scattered L1 sector lookups of the thread form.
constexpr int kInterpTileThreads = 256;

template <typename T, int D, int MM, int START>
__device__ __forceinline__ typename Cplx<T>::type
interp_tile_node(const Geom &g, const T *__restrict__ tab, const typename Cplx<T>::type *tile,
                 const int *st, const int *loc, const T *frac)
{
    using C = typename Cplx<T>::type;
    constexpr int NT = 2 * MM + 1;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    C acc;
    acc.x = (T)0;
    acc.y = (T)0;
    if (D == 1) {
        T w0[NT];
        eval_taps<T, MM, START>(g, tab, 0, frac[0], w0);
        const C *row = tile + loc[0];
#pragma unroll
        for (int i = START; i < NT; i++) {
            const C v = row[i];
            acc.x += v.x * w0[i];
            acc.y += v.y * w0[i];
        }
    } else if (D == 2) {
        T w1[NT];
        eval_taps<T, MM, START>(g, tab + AS, 1, frac[1], w1);
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = eval_tap<T, MM>(g, tab, 0, i0, frac[0]);
            const C *row = tile + (loc[0] + i0) * st[0] + loc[1];
            C in;
            in.x = (T)0;
            in.y = (T)0;
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const C v = row[i1];
                in.x += v.x * w1[i1];
                in.y += v.y * w1[i1];
            }
            acc.x += in.x * w0;
            acc.y += in.y * w0;
        }
    } else {
        T w1[NT], w2[NT];
        eval_taps<T, MM, START>(g, tab + AS, 1, frac[1], w1);
        eval_taps<T, MM, START>(g, tab + 2 * AS, 2, frac[2], w2);
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = eval_tap<T, MM>(g, tab, 0, i0, frac[0]);
            const C *plane = tile + (loc[0] + i0) * st[0];
            C pl;
            pl.x = (T)0;
            pl.y = (T)0;
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const C *row = plane + (loc[1] + i1) * st[1] + loc[2];
                C in;
                in.x = (T)0;
                in.y = (T)0;
#pragma unroll
                for (int i2 = START; i2 < NT; i2++) {
                    const C v = row[i2];
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

template <typename T, int D, int MM>
__global__ void __launch_bounds__(kInterpTileThreads)
    interp_tile_kernel(Geom g, const typename Cplx<T>::type *__restrict__ grid,
                       const typename RecOf<T>::type *__restrict__ rec,
                       const int *__restrict__ perm, const SubProb *__restrict__ subs,
                       const int *__restrict__ nsub_total, typename Cplx<T>::type *__restrict__ f)
{
    using C = typename Cplx<T>::type;
    __shared__ __align__(16) T tab[kMaxDim * poly_axis_stride(sizeof(T) == 8, MM)];
    load_window_tables<T, MM>(tab, g.poly, D);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tile = reinterpret_cast<C *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NWARP = kInterpTileThreads / 32;
    int tdim[D], st[D];
    int cells = 1;
#pragma unroll
    for (int t = 0; t < D; t++) {
        tdim[t] = g.bs[t] + 2 * MM;
        cells *= tdim[t];
    }
    st[D - 1] = 1;
#pragma unroll
    for (int t = D - 2; t >= 0; t--) st[t] = st[t + 1] * tdim[t + 1];
    const int rows = cells / tdim[D - 1];
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
        // stage the tile: cell (a_0..a_{d-1}) holds grid point (origin_t - m + a_t) mod n_t
        for (int row = warp; row < rows; row += NWARP) {
            size_t gbase = 0;
            {
                int rem = row;
                int a[D];
                a[D - 1] = 0;
#pragma unroll
                for (int t = D - 2; t >= 0; t--) {
                    a[t] = rem % tdim[t];
                    rem /= tdim[t];
                }
#pragma unroll
                for (int t = 0; t < D - 1; t++)
                    gbase = gbase * g.n[t] + (size_t)modn(origin[t] - MM + a[t], g.n[t]);
                gbase *= g.n[D - 1];
            }
            for (int a = lane; a < tdim[D - 1]; a += 32)
                tile[row * tdim[D - 1] + a] =
                    grid[gbase + (size_t)modn(origin[D - 1] - MM + a, g.n[D - 1])];
        }
        __syncthreads();
        for (int k = tid; k < P.count; k += kInterpTileThreads) {
            const int s = P.start + k;
            const typename RecOf<T>::type r = rec[s];
            int cell = r.cell;
            int loc[D];
            T frac[D];
            bool edge = false;
#pragma unroll
            for (int t = D - 1; t >= 0; t--) {
                loc[t] = (cell & g.cmask[t]) - origin[t];  // in [0, bs_t)
                cell >>= g.cbits[t];
                frac[t] = r.fr[t];
                edge |= (frac[t] == (T)0);
            }
            const C v = edge ? interp_tile_node<T, D, MM, 0>(g, tab, tile, st, loc, frac)
                             : interp_tile_node<T, D, MM, 1>(g, tab, tile, st, loc, frac);
            f[perm[s]] = v;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------- warp form of B
// One warp per node: the lanes cover the node's taps (last axis fastest, so a warp load touches
// a few contiguous grid rows instead of 32 scattered ones), each per-axis window value is
// evaluated by one lane and broadcast with shuffles, and the partial sums are reduced across
// the warp.
constexpr int kInterpWarps = 8;

template <typename T, int D, int MM, int START>
__device__ __forceinline__ typename Cplx<T>::type
interp_warp_taps(const Geom &g, const typename Cplx<T>::type *__restrict__ grid, const int *base,
                 T wa, T wb, int lane)
{
    using C = typename Cplx<T>::type;
    constexpr int NT = 2 * MM + 1;
    constexpr int NW = D * NT;
    constexpr int PER = NT - START;
    constexpr int TAPS = D == 1 ? PER : (D == 2 ? PER * PER : PER * PER * PER);
    C acc;
    acc.x = (T)0;
    acc.y = (T)0;
#pragma unroll 2
    for (int b0 = 0; b0 < TAPS; b0 += 32) {
        const int q = b0 + lane;
        int rem = q < TAPS ? q : 0;
        T w = (T)1;
        size_t gi = 0;
        size_t stride = 1;
#pragma unroll
        for (int t = D - 1; t >= 0; t--) {
            const int a = rem % PER;
            rem /= PER;
            const int src = t * NT + a + START;
            const T wa_s = __shfl_sync(0xffffffffu, wa, src & 31);
            T wt = wa_s;
            if (NW > 32) {
                const T wb_s = __shfl_sync(0xffffffffu, wb, src & 31);
                wt = src < 32 ? wa_s : wb_s;
            }
            w *= wt;
            gi += (size_t)wrapn(base[t] - MM + a + START, g.n[t]) * stride;
            stride *= (size_t)g.n[t];
        }
        if (q < TAPS) {
            const C v = grid[gi];
            acc.x += v.x * w;
            acc.y += v.y * w;
        }
    }
    return acc;
}

template <typename T, int D, int MM>
__global__ void __launch_bounds__(32 * kInterpWarps)
    interp_warp_kernel(Geom g, const typename Cplx<T>::type *__restrict__ grid,
                       const typename RecOf<T>::type *__restrict__ rec,
                       const int *__restrict__ perm, int M, typename Cplx<T>::type *__restrict__ f)
{
    using C = typename Cplx<T>::type;
    constexpr int NT = 2 * MM + 1;
    constexpr int NW = D * NT;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    __shared__ __align__(16) T tab[kMaxDim * AS];
    load_window_tables<T, MM>(tab, g.poly, D);
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * kInterpWarps + (threadIdx.x >> 5);
    if (s >= M) return;  // the whole warp leaves together
    const typename RecOf<T>::type r = rec[s];
    int base[D];
    T frac[D];
    bool edge;
    decode_node<T, D>(g, r, base, frac, edge);
    T wa = (T)0, wb = (T)0;
    if (lane < NW) {
        const int t = lane / NT, i = lane - (lane / NT) * NT;
        wa = eval_tap<T, MM>(g, tab + t * AS, t, i, frac[t]);
    }
    if (NW > 32 && lane + 32 < NW) {
        const int q = lane + 32, t = q / NT, i = q - (q / NT) * NT;
        wb = eval_tap<T, MM>(g, tab + t * AS, t, i, frac[t]);
    }
    C acc = edge ? interp_warp_taps<T, D, MM, 0>(g, grid, base, wa, wb, lane)
                 : interp_warp_taps<T, D, MM, 1>(g, grid, base, wa, wb, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) f[perm[s]] = acc;
}

// ------------------------------------------------------------------------- node gradient
// Accumulates, per axis t, sum_l g_l dpsibar_t(.) prod_{u != t} psibar_u(.).
template <typename T, int D, int MM, int START>
__device__ __forceinline__ void grad_node(const Geom &g, const T *__restrict__ tab,
                                          const typename Cplx<T>::type *__restrict__ grid,
                                          const int *base, const T *frac,
                                          typename Cplx<T>::type *acc)
{
    using C = typename Cplx<T>::type;
    constexpr int NT = 2 * MM + 1;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
#pragma unroll
    for (int t = 0; t < D; t++) {
        acc[t].x = (T)0;
        acc[t].y = (T)0;
    }
    if (D == 1) {
        const int n0 = g.n[0];
#pragma unroll
        for (int i = START; i < NT; i++) {
            T w, dw;
            eval_tap_d<T, MM>(g, tab, 0, i, frac[0], w, dw);
            const C v = grid[wrapn(base[0] - MM + i, n0)];
            acc[0].x += v.x * dw;
            acc[0].y += v.y * dw;
        }
    } else if (D == 2) {
        T w1[NT], d1[NT];
#pragma unroll
        for (int i = START; i < NT; i++)
            eval_tap_d<T, MM>(g, tab + AS, 1, i, frac[1], w1[i], d1[i]);
        const int n0 = g.n[0], n1 = g.n[1];
        for (int i0 = START; i0 < NT; i0++) {
            T w0, d0;
            eval_tap_d<T, MM>(g, tab, 0, i0, frac[0], w0, d0);
            const C *row = grid + (size_t)wrapn(base[0] - MM + i0, n0) * n1;
            C s0, s1;
            s0.x = s0.y = s1.x = s1.y = (T)0;
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const C v = row[wrapn(base[1] - MM + i1, n1)];
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
#pragma unroll
        for (int i = START; i < NT; i++) {
            eval_tap_d<T, MM>(g, tab + AS, 1, i, frac[1], w1[i], d1[i]);
            eval_tap_d<T, MM>(g, tab + 2 * AS, 2, i, frac[2], w2[i], d2[i]);
        }
        const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
        for (int i0 = START; i0 < NT; i0++) {
            T w0, d0;
            eval_tap_d<T, MM>(g, tab, 0, i0, frac[0], w0, d0);
            const C *plane = grid + (size_t)wrapn(base[0] - MM + i0, n0) * n1 * n2;
            C p0, p1, p2;  // plane sums for the three partial derivatives
            p0.x = p0.y = p1.x = p1.y = p2.x = p2.y = (T)0;
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const C *row = plane + (size_t)wrapn(base[1] - MM + i1, n1) * n2;
                C sw, sd;
                sw.x = sw.y = sd.x = sd.y = (T)0;
#pragma unroll
                for (int i2 = START; i2 < NT; i2++) {
                    const C v = row[wrapn(base[2] - MM + i2, n2)];
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
__global__ void __launch_bounds__(kInterpThreads)
    grad_kernel(Geom g, const __grid_constant__ WinCoef<T, MM> wc,
                const typename Cplx<T>::type *__restrict__ grid,
                const typename RecOf<T>::type *__restrict__ rec, const int *__restrict__ perm,
                int M, const typename Cplx<T>::type *__restrict__ w, T *__restrict__ gx)
{
    const T *tab = wc.c;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const typename RecOf<T>::type r = rec[s];
    int base[D];
    T frac[D];
    bool edge;
    decode_node<T, D>(g, r, base, frac, edge);
    typename Cplx<T>::type acc[D];
    if (!edge)
        grad_node<T, D, MM, 1>(g, tab, grid, base, frac, acc);
    else
        grad_node<T, D, MM, 0>(g, tab, grid, base, frac, acc);
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
                            const SubProb *subs, const int *nsub_total, int max_subs,
                            typename Cplx<T>::type *f, cudaStream_t stream)
{
    using C = typename Cplx<T>::type;
    size_t cells = 1;
    for (int t = 0; t < D; t++) cells *= (size_t)(g.bs[t] + 2 * MM);
    const size_t tile = cells * sizeof(C);
    constexpr size_t tables = kMaxDim * poly_axis_stride(sizeof(T) == 8, MM) * sizeof(T);
    int method = g.interp_method;
    // measured fastest on the GB300: the thread form everywhere (with the nodes of a bin
    // ordered by grid row, the clustered 3-D workload takes 1.08 ms against 1.41 ms for the
    // octet form)
    if (method == kInterpAuto) method = kInterpThread;
    if (method == kInterpTile && tile + tables > 227 * 1024) method = kInterpThread;
    if (method == kInterpTile) {
        cudaError_t e = ensure_dynamic_smem(interp_tile_kernel<T, D, MM>, tile);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, interp_tile_kernel<T, D, MM>,
                                                          kInterpTileThreads, tile);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidValue;
        int blocks = num_sms() * per_sm;
        if (blocks > max_subs) blocks = max_subs;
        interp_tile_kernel<T, D, MM><<<blocks, kInterpTileThreads, tile, stream>>>(
            g, grid, rec, perm, subs, nsub_total, f);
    } else if (method == kInterpOctet && D >= 2 && 2 * MM <= 8) {
        if constexpr (D >= 2 && 2 * MM <= 8) {
            const int64_t blocks = (8 * M + kInterpThreads - 1) / kInterpThreads;
            if (g.lin_k)
                interp_octet_kernel<T, D, MM, true><<<(unsigned)blocks, kInterpThreads, 0,
                                                      stream>>>(g, grid, rec, perm, (int)M, f);
            else
                interp_octet_kernel<T, D, MM, false><<<(unsigned)blocks, kInterpThreads, 0,
                                                       stream>>>(g, grid, rec, perm, (int)M, f);
        }
    } else if (method == kInterpWarp) {
        const int64_t blocks = (M + kInterpWarps - 1) / kInterpWarps;
        interp_warp_kernel<T, D, MM><<<(unsigned)blocks, 32 * kInterpWarps, 0, stream>>>(
            g, grid, rec, perm, (int)M, f);
    } else {
        const int64_t blocks = (M + kInterpThreads - 1) / kInterpThreads;
        if (g.lin_k)
            interp_kernel<T, D, MM, true><<<(unsigned)blocks, kInterpThreads, 0, stream>>>(
                g, make_wincoef<T, MM>(g), grid, rec, perm, (int)M, f);
        else
            interp_kernel<T, D, MM, false><<<(unsigned)blocks, kInterpThreads, 0, stream>>>(
                g, make_wincoef<T, MM>(g), grid, rec, perm, (int)M, f);
    }
    return cudaGetLastError();
}

template <typename T, int D, int MM>
cudaError_t launch_grad_m(const Geom &g, const typename Cplx<T>::type *grid,
                          const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                          const typename Cplx<T>::type *w, T *gx, cudaStream_t stream)
{
    const int64_t blocks = (M + kInterpThreads - 1) / kInterpThreads;
    grad_kernel<T, D, MM><<<(unsigned)blocks, kInterpThreads, 0, stream>>>(
        g, make_wincoef<T, MM>(g), grid, rec, perm, (int)M, w, gx);
    return cudaGetLastError();
}

template <typename T, int D>
cudaError_t interp_d(const Geom &g, const typename Cplx<T>::type *grid,
                     const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                     const SubProb *subs, const int *nsub_total, int max_subs,
                     typename Cplx<T>::type *f, cudaStream_t stream)
{
    GBNFFT_DISPATCH_M(launch_interp_m, T, D, g, grid, rec, perm, M, subs, nsub_total, max_subs,
                      f, stream)
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
