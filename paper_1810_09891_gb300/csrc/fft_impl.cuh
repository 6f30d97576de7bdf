// One axis pass of the d-variate FFT of Algorithm "NFFT" / "adjoint NFFT" (Section 2), with the
// deconvolution D (or D^H) and the zero padding (or cropping) fused in, so that the FFT is
// pruned: a forward transform only ever transforms lines that hold nonzero data, and an adjoint
// transform only writes the |I_N| outputs it needs.
//
// A CTA loads P lines of length L = 2^LOGL of one axis into shared memory, runs a Stockham
// autosort FFT (radix 4, one radix-2 pass when LOGL is odd) entirely in shared memory, and
// writes the lines back. Lines along the contiguous axis are rows; lines along a strided axis
// are taken P columns at a time so that global loads and stores are coalesced. The kernel is
// instantiated per LOGL, so every index of the passes is a compile-time shift or mask; one
// thread owns one radix-4 butterfly per pass (several only for the longest lines).
//
// The deconvolution factor of axis t is applied in the pass of axis t (the factor of
// Algorithm "NFFT" line 2, 1/(|I_n| c_k), is a product over axes). The factors are computed in
// FP64 at plan creation and stored in the plan's precision.
#pragma once

#include "gbnfft_internal.cuh"

namespace gbnfft {

namespace {

template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b)
{
    C r;
    r.x = a.x + b.x;
    r.y = a.y + b.y;
    return r;
}
template <typename C> __device__ __forceinline__ C csub(C a, C b)
{
    C r;
    r.x = a.x - b.x;
    r.y = a.y - b.y;
    return r;
}
// multiply by (INV ? +i : -i)
template <bool INV, typename C> __device__ __forceinline__ C cmul_i(C a)
{
    C r;
    if (!INV) {
        r.x = a.y;
        r.y = -a.x;
    } else {
        r.x = -a.y;
        r.y = a.x;
    }
    return r;
}

// Largest CTA per precision: FP32 lines up to 16384 points use 1024 threads; FP64 lines (up to
// 8192 points) use at most 512 threads so that each thread keeps its values in registers.
template <typename T> struct FftMaxThreads { static constexpr int value = 1024; };
template <> struct FftMaxThreads<double> { static constexpr int value = 512; };

// One Stockham pass of radix 4 (or 2) with stride Ns = 2^LOGNS over the P lines in `s`; each
// thread owns KB radix-4 butterflies' worth of values (KB * 4 / R butterflies of this pass).
template <typename T, int LOGL, int LOGNS, int LOGR, int KB, bool INV>
__device__ __forceinline__ void stockham_pass(typename Cplx<T>::type *s, int pitch, int nbf,
                                              const typename Cplx<T>::type *__restrict__ tw)
{
    using C = typename Cplx<T>::type;
    constexpr int R = 1 << LOGR;
    constexpr int LOGLR = LOGL - LOGR;
    constexpr int LR = 1 << LOGLR;
    constexpr int Ns = 1 << LOGNS;
    constexpr int K = KB * (4 / R);
    const int tid = threadIdx.x, T_ = blockDim.x;
    C v[K][R];
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int b = tid + k * T_;
        if (b < nbf) {
            const int c = b >> LOGLR, j = b & (LR - 1);
#pragma unroll
            for (int r = 0; r < R; r++) v[k][r] = s[c * pitch + j + r * LR];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int b = tid + k * T_;
        if (b < nbf) {
            const int c = b >> LOGLR, j = b & (LR - 1);
            const int kk = j & (Ns - 1);
            const int tws = kk << (LOGL - LOGNS - LOGR);  // twiddle e^{-2 pi i kk/(Ns R)} step
            const int idxD = ((j >> LOGNS) << (LOGNS + LOGR)) + kk;
            C *o = s + c * pitch + idxD;
            if (R == 4) {
                C a0 = v[k][0], a1 = v[k][1], a2 = v[k][2], a3 = v[k][3];
                if (LOGNS > 0) {
                    C w1 = tw[tws], w2 = tw[2 * tws], w3 = tw[3 * tws];
                    if (INV) {
                        w1.y = -w1.y;
                        w2.y = -w2.y;
                        w3.y = -w3.y;
                    }
                    a1 = cmul(a1, w1);
                    a2 = cmul(a2, w2);
                    a3 = cmul(a3, w3);
                }
                // radix-4 DFT with e^{-+2 pi i r s / 4}
                const C t0 = cadd(a0, a2), t1 = csub(a0, a2);
                const C t2 = cadd(a1, a3), t3 = cmul_i<INV>(csub(a1, a3));
                o[0] = cadd(t0, t2);
                o[Ns] = cadd(t1, t3);
                o[2 * Ns] = csub(t0, t2);
                o[3 * Ns] = csub(t1, t3);
            } else {
                C a0 = v[k][0], a1 = v[k][1];
                if (LOGNS > 0) {
                    C w1 = tw[tws];
                    if (INV) w1.y = -w1.y;
                    a1 = cmul(a1, w1);
                }
                o[0] = cadd(a0, a1);
                o[Ns] = csub(a0, a1);
            }
        }
    }
    __syncthreads();
}

template <typename T, int LOGL, int LOGNS, int KB, bool INV>
__device__ __forceinline__ void stockham_all(typename Cplx<T>::type *s, int pitch, int P,
                                             const typename Cplx<T>::type *__restrict__ tw)
{
    if constexpr (LOGNS < LOGL) {
        constexpr int LOGR = (LOGL - LOGNS) >= 2 ? 2 : 1;
        stockham_pass<T, LOGL, LOGNS, LOGR, KB, INV>(s, pitch, P << (LOGL - LOGR), tw);
        stockham_all<T, LOGL, LOGNS + LOGR, KB, INV>(s, pitch, P, tw);
    }
}

template <typename T, int LOGL, int KB>
__global__ void __launch_bounds__(FftMaxThreads<T>::value)
    fft_axis_kernel(const typename Cplx<T>::type *__restrict__ in,
                    typename Cplx<T>::type *__restrict__ out, long long outer, long long inner,
                    int Nt, int P, int pad_mode, int inverse,
                    const typename Cplx<T>::type *__restrict__ tw, const T *__restrict__ deconv)
{
    using C = typename Cplx<T>::type;
    constexpr int L = 1 << LOGL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int pitch = L + 1;
    const int tid = threadIdx.x;
    const int T_ = blockDim.x;
    const int Lin = pad_mode ? Nt : L;
    const int Lout = pad_mode ? L : Nt;
    const int half = Nt / 2;

    // Tile of P lines (P a power of two): contiguous axis -> P consecutive rows; strided axis ->
    // P consecutive columns (inner indices) of one outer index.
    long long o0, i0;
    int lines;
    if (inner == 1) {
        o0 = (long long)blockIdx.x * P;
        i0 = 0;
        lines = (int)min((long long)P, outer - o0);
    } else {
        const long long tiles_per_outer = (inner + P - 1) / P;
        o0 = blockIdx.x / tiles_per_outer;
        i0 = (blockIdx.x - o0 * tiles_per_outer) * P;
        lines = (int)min((long long)P, inner - i0);
    }
    const int logP = __ffs(P) - 1;

    // ---- load (zero padding + deconvolution in pad mode)
    if (pad_mode) {
        C z;
        z.x = (T)0;
        z.y = (T)0;
        for (int e = tid; e < P * pitch; e += T_) s[e] = z;
        __syncthreads();
    }
    if (inner == 1) {
        for (int c = 0; c < lines; c++) {
            const C *src = in + (o0 + c) * Lin;
            for (int p = tid; p < Lin; p += T_) {
                C v = src[p];
                int pos = p;
                if (pad_mode) {
                    const T w = deconv[p];
                    v.x *= w;
                    v.y *= w;
                    pos = p - half;
                    if (pos < 0) pos += L;
                }
                s[c * pitch + pos] = v;
            }
        }
    } else {
        const C *src = in + o0 * Lin * inner + i0;
        for (int e = tid; e < (Lin << logP); e += T_) {
            const int p = e >> logP;
            const int c = e & (P - 1);
            if (c >= lines) continue;
            C v = src[(long long)p * inner + c];
            int pos = p;
            if (pad_mode) {
                const T w = deconv[p];
                v.x *= w;
                v.y *= w;
                pos = p - half;
                if (pos < 0) pos += L;
            }
            s[c * pitch + pos] = v;
        }
    }
    __syncthreads();

    // ---- Stockham passes in shared memory (each pass ends with a barrier)
    if (inverse)
        stockham_all<T, LOGL, 0, KB, true>(s, pitch, P, tw);
    else
        stockham_all<T, LOGL, 0, KB, false>(s, pitch, P, tw);

    // ---- store (cropping + deconvolution in crop mode)
    if (inner == 1) {
        for (int c = 0; c < lines; c++) {
            C *dst = out + (o0 + c) * Lout;
            for (int p = tid; p < Lout; p += T_) {
                C v;
                if (pad_mode) {
                    v = s[c * pitch + p];
                } else {
                    int pos = p - half;
                    if (pos < 0) pos += L;
                    v = s[c * pitch + pos];
                    const T w = deconv[p];
                    v.x *= w;
                    v.y *= w;
                }
                dst[p] = v;
            }
        }
    } else {
        C *dst = out + o0 * Lout * inner + i0;
        for (int e = tid; e < (Lout << logP); e += T_) {
            const int p = e >> logP;
            const int c = e & (P - 1);
            if (c >= lines) continue;
            C v;
            if (pad_mode) {
                v = s[c * pitch + p];
            } else {
                int pos = p - half;
                if (pos < 0) pos += L;
                v = s[c * pitch + pos];
                const T w = deconv[p];
                v.x *= w;
                v.y *= w;
            }
            dst[(long long)p * inner + c] = v;
        }
    }
}

template <typename T, int LOGL, int KB>
cudaError_t launch_kb(const typename Cplx<T>::type *in, typename Cplx<T>::type *out,
                      int64_t outer, int64_t inner, int Nt, int P, bool pad_mode, int sign,
                      const typename Cplx<T>::type *twiddle, const T *deconv,
                      cudaStream_t stream)
{
    using C = typename Cplx<T>::type;
    constexpr int L = 1 << LOGL;
    int threads = ((P * L / 4 + KB - 1) / KB + 31) / 32 * 32;
    if (threads < 32) threads = 32;
    if (threads > FftMaxThreads<T>::value) return cudaErrorInvalidValue;
    const size_t smem = (size_t)P * (L + 1) * sizeof(C);
    long long blocks;
    if (inner == 1)
        blocks = (outer + P - 1) / P;
    else
        blocks = outer * ((inner + P - 1) / P);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = ensure_dynamic_smem(fft_axis_kernel<T, LOGL, KB>, smem);
        if (e != cudaSuccess) return e;
    }
    fft_axis_kernel<T, LOGL, KB><<<(unsigned)blocks, threads, smem, stream>>>(
        in, out, outer, inner, Nt, P, pad_mode ? 1 : 0, sign > 0 ? 1 : 0, twiddle, deconv);
    return cudaGetLastError();
}

template <typename T, int LOGL>
cudaError_t launch_fixed(const typename Cplx<T>::type *in, typename Cplx<T>::type *out,
                         int64_t outer, int64_t inner, int Nt, bool pad_mode, int sign,
                         const typename Cplx<T>::type *twiddle, const T *deconv,
                         cudaStream_t stream)
{
    using C = typename Cplx<T>::type;
    constexpr int L = 1 << LOGL;
    // Lines per CTA (a power of two): 1 along the contiguous axis; along a strided axis enough
    // columns for a 32-byte run per row (4 FP32 / 2 FP64 complex values), so that loads and
    // stores use whole sectors. Short lines widen the tile (up to 1024 points) while the grid
    // keeps at least four CTAs per SM. Threads: one radix-4 butterfly each (KB = 1) for tiles of
    // up to 2048 points, else four (KB = 4), which keeps CTAs small enough for several per SM.
    const int64_t lines = outer * inner;
    const int64_t min_ctas = 4 * (int64_t)num_sms();
    int P = 1;
    if (inner > 1) P = (int)(32 / sizeof(C));
    while (P * L < 1024 && lines / (2 * P) >= min_ctas) P *= 2;
    const int64_t cap = inner > 1 ? inner : outer;
    while (P > 1 && P > cap) P /= 2;
    while (P > 1 && (int64_t)P * L / 16 > FftMaxThreads<T>::value) P /= 2;
    if ((int64_t)P * L <= 2048)
        return launch_kb<T, LOGL, 1>(in, out, outer, inner, Nt, P, pad_mode, sign, twiddle,
                                     deconv, stream);
    return launch_kb<T, LOGL, 4>(in, out, outer, inner, Nt, P, pad_mode, sign, twiddle, deconv,
                                 stream);
}

}  // namespace

template <typename T>
cudaError_t launch_fft_axis(const typename Cplx<T>::type *in, typename Cplx<T>::type *out,
                            int64_t outer, int64_t inner, int L, int Nt, bool pad_mode, int sign,
                            const typename Cplx<T>::type *twiddle, const T *deconv,
                            cudaStream_t stream)
{
    if (outer <= 0 || inner <= 0) return cudaSuccess;
    if (L < 2 || (L & (L - 1)) != 0) return cudaErrorInvalidValue;
#define GB_FFT_CASE(LG)                                                                            \
    case LG:                                                                                      \
        return launch_fixed<T, LG>(in, out, outer, inner, Nt, pad_mode, sign, twiddle, deconv,   \
                                   stream);
    switch (__builtin_ctz((unsigned)L)) {
        GB_FFT_CASE(1)
        GB_FFT_CASE(2)
        GB_FFT_CASE(3)
        GB_FFT_CASE(4)
        GB_FFT_CASE(5)
        GB_FFT_CASE(6)
        GB_FFT_CASE(7)
        GB_FFT_CASE(8)
        GB_FFT_CASE(9)
        GB_FFT_CASE(10)
        GB_FFT_CASE(11)
        GB_FFT_CASE(12)
        GB_FFT_CASE(13)
        GB_FFT_CASE(14)
    default: return cudaErrorInvalidValue;
    }
#undef GB_FFT_CASE
}

}  // namespace gbnfft
