// Window evaluation in grid units, normalised to psibar(0) = 1 (Section 2, eq. window and
// eq. window_cutoff). The default window is Kaiser-Bessel,
//
//   psi(t) = sinh(b u) / (pi u),  u = sqrt(m^2 - t^2),  |t| <= m;  psi(t) = 0 for |t| > m,
//
// (the pair of Plonka-Potts-Steidl-Tasche Ch. 7.2); Gaussian, B-spline and sinc windows
// (Section 4.1) go through the same code. The factor psi(0) moves into the deconvolution
// table, so sums of products of d weights stay in range in FP32 for every m. A node with
// offset frac has taps t = frac + m - i, i = 0..2m; i = 0 lies inside the closed support only
// when frac == 0 (value psibar(m), a per-axis constant). For i = 1..2m the kernels evaluate
// psibar(frac + m - i) from a per-tap polynomial in frac: each window is smooth on every tap
// interval (the B-spline is a polynomial of degree 2m - 1 there), so low degrees suffice; the
// polynomials are fitted on the host at plan creation (see gbnfft_internal.cuh).
#pragma once

#include <cuda_runtime.h>

#include "gbnfft_internal.cuh"

namespace gbnfft {

// ------------------------------------------------------------------------ polynomial form
template <typename T, int MM> struct PolyDeg {
    static constexpr int value = poly_degree(sizeof(T) == 8, MM);
};

// All taps of one axis: w[i] = psibar(frac + m - i) for i = START..2m. c is the axis' table
// (shared, constant or global memory); w[0] (START = 0) is the edge tap, nonzero only when
// frac == 0. Taps i and 2m + 1 - i mirror each other: psibar is even, so their functions of z
// are f_i(z) and f_i(-z), and the Chebyshev interpolants, fitted at nodes symmetric about 0,
// satisfy P_(2m+1-i)(z) = P_i(-z). With P_i(z) = E_i(z^2) + z O_i(z^2) (the even- and
// odd-degree coefficients) one pair costs about one Horner evaluation:
// w[i] = E + z O, w[2m + 1 - i] = E - z O.
template <typename T, int MM, int START>
__device__ __forceinline__ void window_taps(const T *__restrict__ c, T frac, T edge_w, T *w)
{
    constexpr int DEG = PolyDeg<T, MM>::value;
    constexpr int KE = DEG - (DEG & 1);        // highest even degree
    constexpr int KO = DEG - 1 + (DEG & 1);    // highest odd degree
    const T z = (T)2 * frac - (T)1;
    const T u = z * z;
    T e[MM], o[MM];
#pragma unroll
    for (int i = 1; i <= MM; i++) {
        e[i - 1] = c[KE * kPolyTaps + i - 1];
        o[i - 1] = c[KO * kPolyTaps + i - 1];
    }
#pragma unroll
    for (int k = KE - 2; k >= 0; k -= 2) {
#pragma unroll
        for (int i = 1; i <= MM; i++) e[i - 1] = fma(e[i - 1], u, c[k * kPolyTaps + i - 1]);
    }
#pragma unroll
    for (int k = KO - 2; k >= 1; k -= 2) {
#pragma unroll
        for (int i = 1; i <= MM; i++) o[i - 1] = fma(o[i - 1], u, c[k * kPolyTaps + i - 1]);
    }
#pragma unroll
    for (int i = 1; i <= MM; i++) {
        w[i] = fma(z, o[i - 1], e[i - 1]);
        w[2 * MM + 1 - i] = fma(-z, o[i - 1], e[i - 1]);
    }
    if (START == 0) w[0] = frac == (T)0 ? edge_w : (T)0;
}

// One tap i (0..2m) of one axis.
template <typename T, int MM>
__device__ __forceinline__ T window_tap(const T *__restrict__ c, int i, T frac, T edge_w)
{
    constexpr int DEG = PolyDeg<T, MM>::value;
    if (i == 0) return frac == (T)0 ? edge_w : (T)0;
    const T z = (T)2 * frac - (T)1;
    T acc = c[DEG * kPolyTaps + i - 1];
#pragma unroll
    for (int k = DEG - 1; k >= 0; k--) acc = fma(acc, z, c[k * kPolyTaps + i - 1]);
    return acc;
}

// Value and t-derivative of one tap: d psibar / dt = d P / d frac = 2 dP/dz.
template <typename T, int MM>
__device__ __forceinline__ void window_tap_d(const T *__restrict__ c, int i, T frac, T edge_w,
                                             T edge_dw, T &w, T &dw)
{
    constexpr int DEG = PolyDeg<T, MM>::value;
    if (i == 0) {
        const bool on = frac == (T)0;
        w = on ? edge_w : (T)0;
        dw = on ? edge_dw : (T)0;
        return;
    }
    const T z = (T)2 * frac - (T)1;
    T p = c[DEG * kPolyTaps + i - 1], dp = (T)0;
#pragma unroll
    for (int k = DEG - 1; k >= 0; k--) {
        dp = fma(dp, z, p);
        p = fma(p, z, c[k * kPolyTaps + i - 1]);
    }
    w = p;
    dw = (T)2 * dp;
}

// Horner evaluation with the coefficients in registers (c[0..DEG], lowest degree first).
template <typename T, int DEG>
__device__ __forceinline__ T poly_horner(const T *c, T z)
{
    T acc = c[DEG];
#pragma unroll
    for (int k = DEG - 1; k >= 0; k--) acc = fma(acc, z, c[k]);
    return acc;
}

// Tap i (1..2m) of one axis from a table in shared memory (c = the axis' table).
template <typename T, int DEG>
__device__ __forceinline__ T poly_horner_tap(const T *c, int i, T z)
{
    T acc = c[DEG * kPolyTaps + i - 1];
#pragma unroll
    for (int k = DEG - 1; k >= 0; k--) acc = fma(acc, z, c[k * kPolyTaps + i - 1]);
    return acc;
}

// ------------------------------------------------------------------- lookup table (PRE_LIN_PSI)
// With NFFT_OPT_WINDOW_TABLE = K the window comes from a table of psibar at K points per unit
// of t, linearly interpolated (Section 3.1, Table tab:nfftflags, PRE_LIN_PSI). The table of an
// axis is laid out per offset sample: lt[j * 2m + (i - 1)] = psibar(j / K + m - i) for tap
// i = 1..2m and j = 0..K, so that the 2m taps of a node share one interpolation position
// frac * K and read two runs of 2m neighbouring values. The derivative at a sample is the
// slope of the segment above it (the right derivative in t).
template <typename T>
__device__ __forceinline__ void lin_pos(T frac, int K, int &j, T &lam)
{
    const T u = frac * (T)K;  // frac in [0, 1]
    j = (int)u;
    if (j > K - 1) j = K - 1;
    lam = u - (T)j;
}

template <typename T, int MM>
__device__ __forceinline__ T lin_at(const T *__restrict__ lt, int j, T lam, int i)
{
    const T a = lt[j * (2 * MM) + i - 1], b = lt[(j + 1) * (2 * MM) + i - 1];
    return fma(lam, b - a, a);
}

// All taps of one axis (as window_taps).
template <typename T, int MM, int START>
__device__ __forceinline__ void lin_taps(const T *__restrict__ lt, int K, T frac, T edge_w, T *w)
{
    int j;
    T lam;
    lin_pos(frac, K, j, lam);
#pragma unroll
    for (int i = 1; i <= 2 * MM; i++) w[i] = lin_at<T, MM>(lt, j, lam, i);
    if (START == 0) w[0] = frac == (T)0 ? edge_w : (T)0;
}

// One tap i (0..2m) of one axis (as window_tap).
template <typename T, int MM>
__device__ __forceinline__ T lin_tap(const T *__restrict__ lt, int K, int i, T frac, T edge_w)
{
    if (i == 0) return frac == (T)0 ? edge_w : (T)0;
    int j;
    T lam;
    lin_pos(frac, K, j, lam);
    return lin_at<T, MM>(lt, j, lam, i);
}

// Value and t-derivative of one tap (as window_tap_d; edge_dw is the plan's edge slope).
template <typename T, int MM>
__device__ __forceinline__ void lin_tap_d(const T *__restrict__ lt, int K, int i, T frac,
                                          T edge_w, T edge_dw, T &w, T &dw)
{
    if (i == 0) {
        const bool on = frac == (T)0;
        w = on ? edge_w : (T)0;
        dw = on ? edge_dw : (T)0;
        return;
    }
    int j;
    T lam;
    lin_pos(frac, K, j, lam);
    const T a = lt[j * (2 * MM) + i - 1], b = lt[(j + 1) * (2 * MM) + i - 1];
    w = fma(lam, b - a, a);
    dw = (b - a) * (T)K;
}

// Axis t's table inside the plan's table block.
template <typename T, int MM>
__device__ __forceinline__ const T *lin_axis(const void *lin, int K, int t)
{
    return static_cast<const T *>(lin) + (size_t)t * (K + 1) * (2 * MM);
}

// Window evaluation on axis t of a plan: the lookup table when the plan has one (g.lin_k > 0),
// else the per-tap polynomials `poly` of that axis. MODE 0 decides at run time (a uniform
// branch); kernels instantiated per evaluation pass MODE 1 (polynomials) or 2 (table).
template <int MODE> __device__ __forceinline__ bool use_table(const Geom &g)
{
    return MODE == 2 || (MODE == 0 && g.lin_k > 0);
}

template <typename T, int MM, int START, int MODE = 0>
__device__ __forceinline__ void eval_taps(const Geom &g, const T *__restrict__ poly, int t, T frac,
                                          T *w)
{
    if (use_table<MODE>(g))
        lin_taps<T, MM, START>(lin_axis<T, MM>(g.lin, g.lin_k, t), g.lin_k, frac,
                               (T)g.win[t].edge_w, w);
    else
        window_taps<T, MM, START>(poly, frac, (T)g.win[t].edge_w, w);
}

template <typename T, int MM, int MODE = 0>
__device__ __forceinline__ T eval_tap(const Geom &g, const T *__restrict__ poly, int t, int i,
                                      T frac)
{
    if (use_table<MODE>(g))
        return lin_tap<T, MM>(lin_axis<T, MM>(g.lin, g.lin_k, t), g.lin_k, i, frac,
                              (T)g.win[t].edge_w);
    return window_tap<T, MM>(poly, i, frac, (T)g.win[t].edge_w);
}

template <typename T, int MM, int MODE = 0>
__device__ __forceinline__ void eval_tap_d(const Geom &g, const T *__restrict__ poly, int t, int i,
                                           T frac, T &w, T &dw)
{
    if (use_table<MODE>(g))
        lin_tap_d<T, MM>(lin_axis<T, MM>(g.lin, g.lin_k, t), g.lin_k, i, frac, (T)g.win[t].edge_w,
                         (T)g.win[t].edge_dw, w, dw);
    else
        window_tap_d<T, MM>(poly, i, frac, (T)g.win[t].edge_w, (T)g.win[t].edge_dw, w, dw);
}

// Copy the window tables (d axes) into shared memory; every thread of the CTA must call it.
template <typename T, int MM>
__device__ __forceinline__ void load_window_tables(T *dst, const void *src, int d)
{
    const T *s = static_cast<const T *>(src);
    const int n = d * poly_axis_stride(sizeof(T) == 8, MM);
    for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = s[e];
    __syncthreads();
}

}  // namespace gbnfft
