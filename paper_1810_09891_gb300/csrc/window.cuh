// Kaiser-Bessel window in grid units, normalised to psibar(0) = 1 (Section 2, eq. window and
// eq. window_cutoff; the pair itself is the one of Plonka-Potts-Steidl-Tasche Ch. 7.2):
//
//   psi(t)    = sinh(b u) / (pi u),  u = sqrt(m^2 - t^2),  |t| <= m;  psi(t) = 0 for |t| > m,
//   psibar(t) = psi(t) / psi(0) = kscale * sinh(b u) / u,  kscale = m / sinh(b m).
//
// The factor psi(0) moves into the deconvolution table, so sums of products of d weights stay
// in range in FP32 for every m. Each tap evaluates the window at t = frac + m - i for
// i = 0..2m; m^2 - t^2 is formed as (i - frac)(2m - i + frac), which has no cancellation near
// the support edge. i = 0 lies inside the closed support only when frac == 0.
#pragma once

#include <cuda_runtime.h>

namespace gbnfft {

__device__ __forceinline__ float kb_sinh(float z) { return sinhf(z); }
__device__ __forceinline__ double kb_sinh(double z) { return sinh(z); }
__device__ __forceinline__ float kb_cosh(float z) { return coshf(z); }
__device__ __forceinline__ double kb_cosh(double z) { return cosh(z); }
__device__ __forceinline__ float kb_sqrt(float z) { return sqrtf(z); }
__device__ __forceinline__ double kb_sqrt(double z) { return sqrt(z); }

// psibar at tap i of a node with offset frac (t = frac + m - i).
template <typename T>
__device__ __forceinline__ T psibar_tap(int i, int m, T frac, T b, T kscale)
{
    const T s = ((T)i - frac) * ((T)(2 * m - i) + frac);  // m^2 - t^2
    if (s > (T)0) {
        const T u = kb_sqrt(s);
        return kscale * kb_sinh(b * u) / u;
    }
    return s == (T)0 ? kscale * b : (T)0;  // limit sinh(b u)/u -> b at the edge
}

// d psibar / dt at tap i:  -kscale * t * (b u cosh(b u) - sinh(b u)) / u^3.
// For small z = b u the bracket over u^3 is b^3/3 (1 + z^2/10 + z^4/280 + z^6/15120) (its
// Taylor series); the switch point keeps both branches accurate in the given precision.
template <typename T> struct DpsiSwitch;
template <> struct DpsiSwitch<float> { static constexpr float z = 0.5f; };
template <> struct DpsiSwitch<double> { static constexpr double z = 0.05; };

template <typename T>
__device__ __forceinline__ T dpsibar_tap(int i, int m, T frac, T b, T kscale)
{
    const T s = ((T)i - frac) * ((T)(2 * m - i) + frac);
    if (s < (T)0) return (T)0;
    const T t = (T)(m - i) + frac;
    const T u = kb_sqrt(s);
    const T z = b * u;
    T g;
    if (z < DpsiSwitch<T>::z) {
        const T z2 = z * z;
        g = b * b * b / (T)3 *
            ((T)1 + z2 * ((T)0.1 + z2 * ((T)1 / (T)280 + z2 * ((T)1 / (T)15120))));
    } else {
        g = (z * kb_cosh(z) - kb_sinh(z)) / (u * u * u);
    }
    return -kscale * t * g;
}

}  // namespace gbnfft
