// One axis pass of the d-variate FFT of Algorithm "NFFT" / "adjoint NFFT" (Section 2), with the
// deconvolution D (or D^H) and the zero padding (or cropping) fused in, so that the FFT is
// pruned: a forward transform only ever transforms lines that hold nonzero data, and an adjoint
// transform only writes the |I_N| outputs it needs.
//
// Two line kernels, both instantiated per LOGL (L = 2^LOGL) so that every index is a
// compile-time shift or mask:
//  * fftr_axis_kernel (lines of 16 ... 8192 points in FP32, 16 ... 4096 in FP64): radix-8
//    Stockham stages with the butterflies in registers; the first stage reads global memory and
//    the last one writes it, the stages in between exchange through shared memory.
//  * fft_axis_kernel (all other lengths): a CTA loads P lines into shared memory, runs a
//    radix-4 Stockham FFT (one radix-2 pass when LOGL is odd) there and writes the lines back.
// Lines along the contiguous axis are rows; lines along a strided axis are taken P columns at a
// time so that global loads and stores are coalesced.
//
// The deconvolution factor of axis t is applied in the pass of axis t (the factor
// 1/(|I_n| c_k) of the deconvolution step of Algorithm "NFFT" is a product over axes). The
// factors are computed in FP64 at plan creation and stored in the plan's precision.
#pragma once

#include <algorithm>

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
                      int64_t outer, int64_t inner, int Nt, int P, int pad_mode, int sign,
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
        in, out, outer, inner, Nt, P, pad_mode, sign > 0 ? 1 : 0, twiddle, deconv);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ DFTs in registers
// cos and sin of 2 pi k / 32 for k = 0..15 (DFTs of length <= 32 need no others)
__device__ constexpr double kRootCos[16] = {
    1.0, 0.98078528040323043, 0.92387953251128674, 0.83146961230254524,
    0.70710678118654757, 0.55557023301960229, 0.38268343236508984, 0.19509032201612833,
    0.0, -0.19509032201612833, -0.38268343236508984, -0.55557023301960229,
    -0.70710678118654757, -0.83146961230254524, -0.92387953251128674, -0.98078528040323043};
__device__ constexpr double kRootSin[16] = {
    0.0, 0.19509032201612833, 0.38268343236508984, 0.55557023301960229,
    0.70710678118654757, 0.83146961230254524, 0.92387953251128674, 0.98078528040323043,
    1.0, 0.98078528040323043, 0.92387953251128674, 0.83146961230254524,
    0.70710678118654757, 0.55557023301960229, 0.38268343236508984, 0.19509032201612833};

__host__ __device__ constexpr int bit_reverse(int x, int bits)
{
    int r = 0;
    for (int i = 0; i < bits; i++) r = (r << 1) | ((x >> i) & 1);
    return r;
}

// In-register DFT of length R = 2^LOGR <= 32 (natural order in and out), radix-2 decimation in
// time; every index and twiddle is a compile-time constant once unrolled.
template <typename C, int LOGR, bool INV> __device__ __forceinline__ void dft_reg(C *v)
{
    using T = decltype(v[0].x);
    constexpr int R = 1 << LOGR;
    C a[R];
#pragma unroll
    for (int i = 0; i < R; i++) a[bit_reverse(i, LOGR)] = v[i];
#pragma unroll
    for (int s = 1; s <= LOGR; s++) {
        const int m = 1 << s, h = m >> 1;
#pragma unroll
        for (int k = 0; k < R; k += m) {
#pragma unroll
            for (int j = 0; j < h; j++) {
                const int e = j * (32 / m);  // root index: e^(-+2 pi i j / m) = root32^e
                C b = a[k + j + h];
                if (e == 8) {
                    b = cmul_i<INV>(b);
                } else if (e != 0) {
                    C w;
                    w.x = (T)kRootCos[e];
                    w.y = INV ? (T)kRootSin[e] : -(T)kRootSin[e];
                    b = cmul(b, w);
                }
                const C u = a[k + j];
                a[k + j] = cadd(u, b);
                a[k + j + h] = csub(u, b);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < R; i++) v[i] = a[i];
}

// ---------------------------------------------------------------- radix-8 register Stockham
// The same line transform as the shared-memory Stockham kernel above, with the butterflies in
// registers: stages of radix 8 (the last one of radix 4 or 2 when log2 L is not a multiple of
// 3), L / 8 threads per line, each owning one radix-8 butterfly (or several smaller ones) per
// stage. The first stage reads the line straight from global memory (zero padding and the
// deconvolution factor on the way in), the last one writes it straight back (cropping and the
// factor on the way out); the stages in between exchange through two shared-memory buffers used
// in turn, so one barrier separates consecutive stages. Shared indices are padded by one cell
// per 16, which keeps the stride-8 writes of the first stages free of bank conflicts.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

constexpr int kFftLogR = 3;  // largest stage radix 2^kFftLogR (radix 4 measured slower)
constexpr int kFftR = 1 << kFftLogR;

struct LineIO {
    int Nt, half, pad_mode;
    long long es;
};

template <typename T, int LOGL>
__device__ __forceinline__ typename Cplx<T>::type line_load(const typename Cplx<T>::type *src,
                                                            const LineIO &io, const T *deconv,
                                                            int pos, bool live)
{
    using C = typename Cplx<T>::type;
    constexpr int L = 1 << LOGL;
    C x;
    x.x = (T)0;
    x.y = (T)0;
    if (!live) return x;
    if (io.pad_mode == 1) {
        const int p = (pos + io.half) & (L - 1);
        if (p < io.Nt) {
            x = src[(long long)p * io.es];
            const T w = deconv[p];
            x.x *= w;
            x.y *= w;
        }
    } else {
        x = src[(long long)pos * io.es];
    }
    return x;
}

template <typename T, int LOGL>
__device__ __forceinline__ void line_store(typename Cplx<T>::type *dst, const LineIO &io,
                                           const T *deconv, int pos,
                                           typename Cplx<T>::type y, bool live)
{
    constexpr int L = 1 << LOGL;
    if (!live) return;
    if (io.pad_mode != 0) {  // zero padding or plain: every output
        dst[(long long)pos * io.es] = y;
    } else {
        const int p = (pos + io.half) & (L - 1);
        if (p < io.Nt) {
            const T w = deconv[p];
            y.x *= w;
            y.y *= w;
            dst[(long long)p * io.es] = y;
        }
    }
}

template <typename T, int LOGL, int LOGNS, bool INV>
__device__ __forceinline__ void r8_stage(const typename Cplx<T>::type *src,
                                         typename Cplx<T>::type *dst, const LineIO &io,
                                         const T *deconv, bool live, int j,
                                         typename Cplx<T>::type *bin,
                                         typename Cplx<T>::type *bout,
                                         const typename Cplx<T>::type *__restrict__ tw)
{
    using C = typename Cplx<T>::type;
    constexpr int L = 1 << LOGL;
    constexpr int TL = L / kFftR;
    constexpr int LOGRS = (LOGL - LOGNS) >= kFftLogR ? kFftLogR : (LOGL - LOGNS);
    constexpr int RS = 1 << LOGRS;
    constexpr int K = kFftR / RS;
    constexpr int NS = 1 << LOGNS;
    constexpr bool FIRST = LOGNS == 0;
    constexpr bool LAST = LOGNS + LOGRS == LOGL;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int b = j + k * TL;
        C a[RS];
#pragma unroll
        for (int r = 0; r < RS; r++) {
            const int i = b + r * (L / RS);
            a[r] = FIRST ? line_load<T, LOGL>(src, io, deconv, i, live) : bin[pad16(i)];
        }
        const int kk = b & (NS - 1);
        if (LOGNS > 0) {
#pragma unroll
            for (int r = 1; r < RS; r++) {
                C w = tw[(r * kk) << (LOGL - LOGNS - LOGRS)];
                if (INV) w.y = -w.y;
                a[r] = cmul(a[r], w);
            }
        }
        dft_reg<C, LOGRS, INV>(a);
        const int idx = ((b >> LOGNS) << (LOGNS + LOGRS)) + kk;
#pragma unroll
        for (int r = 0; r < RS; r++) {
            if (LAST)
                line_store<T, LOGL>(dst, io, deconv, idx + r * NS, a[r], live);
            else
                bout[pad16(idx + r * NS)] = a[r];
        }
    }
    if constexpr (!LAST) {
        __syncthreads();
        r8_stage<T, LOGL, LOGNS + LOGRS, INV>(src, dst, io, deconv, live, j, bout, bin, tw);
    }
}

// One CTA's lines of a pass: P lines of L = 2^LOGL points (P * L / 8 threads, `block` the
// CTA's index within the pass, S its shared memory: P line buffers of LS cells).
template <typename T, int LOGL, bool INV>
__device__ __forceinline__ void fftr_block(const typename Cplx<T>::type *__restrict__ in,
                                           typename Cplx<T>::type *__restrict__ out,
                                           long long outer, long long inner, int Nt, int P,
                                           int LS, int pad_mode,
                                           const typename Cplx<T>::type *__restrict__ tw,
                                           const T *__restrict__ deconv, long long block,
                                           typename Cplx<T>::type *S)
{
    using C = typename Cplx<T>::type;
    constexpr int L = 1 << LOGL;
    constexpr int TL = L / kFftR;
    constexpr int BUF = L + L / 16;
    const int tid = threadIdx.x;
    const int Lin = pad_mode == 1 ? Nt : L;
    const int Lout = pad_mode == 0 ? Nt : L;
    int c, j;
    long long o0, i0;
    int lines;
    if (inner == 1) {
        c = tid / TL;
        j = tid - c * TL;
        o0 = block * P;
        i0 = 0;
        lines = (int)min((long long)P, outer - o0);
    } else {
        c = tid % P;
        j = tid / P;
        const long long tiles = (inner + P - 1) / P;
        o0 = block / tiles;
        i0 = (block - o0 * tiles) * P;
        lines = (int)min((long long)P, inner - i0);
    }
    const bool live = c < lines;
    LineIO io;
    io.Nt = Nt;
    io.half = Nt / 2;
    io.pad_mode = pad_mode;
    const C *src;
    C *dst;
    if (inner == 1) {
        src = in + (o0 + c) * Lin;
        dst = out + (o0 + c) * Lout;
        io.es = 1;
    } else {
        src = in + o0 * Lin * inner + i0 + c;
        dst = out + o0 * Lout * inner + i0 + c;
        io.es = inner;
    }
    C *b0 = S + (size_t)c * LS;
    C *b1 = b0 + BUF;
    r8_stage<T, LOGL, 0, INV>(src, dst, io, deconv, live, j, b1, b0, tw);
}

template <typename T, int LOGL, bool INV>
__global__ void __launch_bounds__(FftMaxThreads<T>::value)
    fftr_axis_kernel(const typename Cplx<T>::type *__restrict__ in,
                     typename Cplx<T>::type *__restrict__ out, long long outer, long long inner,
                     int Nt, int P, int LS, int pad_mode,
                     const typename Cplx<T>::type *__restrict__ tw, const T *__restrict__ deconv)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // Launched as a programmatic dependent of the stream's previous kernel: wait here, before
    // any memory access, until that kernel has finished and its writes are visible.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    fftr_block<T, LOGL, INV>(in, out, outer, inner, Nt, P, LS, pad_mode, tw, deconv,
                             (long long)blockIdx.x, reinterpret_cast<C *>(smem_raw));
}

template <typename T, int LOGL>
cudaError_t launch_fftr(const typename Cplx<T>::type *in, typename Cplx<T>::type *out,
                        int64_t outer, int64_t inner, int Nt, int pad_mode, int sign,
                        const typename Cplx<T>::type *twiddle, const T *deconv,
                        cudaStream_t stream)
{
    using C = typename Cplx<T>::type;
    constexpr int L = 1 << LOGL;
    constexpr int TL = L / kFftR;
    const int64_t lines = outer * inner;
    const int64_t min_ctas = 2 * (int64_t)num_sms();
    int P = inner > 1 ? (int)(32 / sizeof(C)) : 1;
    while (P * TL < 256 && lines / (2 * P) >= min_ctas) P *= 2;
    while (P > 1 && P * TL > FftMaxThreads<T>::value) P /= 2;
    const int64_t cap = inner > 1 ? inner : outer;
    while (P > 1 && P > cap) P /= 2;
    if (TL > FftMaxThreads<T>::value) return cudaErrorInvalidValue;
    int LS = 2 * (L + L / 16);
    if (inner > 1 && P > 1) {
        const int cells = 128 / (int)sizeof(C);
        const int want = (cells / P) % cells;
        LS += ((want - LS % cells) + cells) % cells;
    }
    const size_t smem = (size_t)P * LS * sizeof(C);
    long long blocks = inner == 1 ? (outer + P - 1) / P : outer * ((inner + P - 1) / P);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int threads = P * TL;
    // Programmatic dependent launch: the pass is set up and its CTAs made resident while the
    // stream's previous kernel (usually the other pass of the same transform) drains; the
    // kernel waits for it before touching memory. The passes are latency bound, so the hidden
    // launch is a large part of their time (radial 1024^2 step: adjoint 21.3 -> 16.8 us,
    // forward 21.6 -> 19 us).
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const long long outer_ll = outer, inner_ll = inner;
    cudaError_t e;
    if (sign > 0) {
        e = ensure_dynamic_smem(fftr_axis_kernel<T, LOGL, true>, smem);
        if (e != cudaSuccess) return e;
        return cudaLaunchKernelEx(&cfg, fftr_axis_kernel<T, LOGL, true>, in, out, outer_ll,
                                  inner_ll, Nt, P, LS, pad_mode, twiddle, deconv);
    }
    e = ensure_dynamic_smem(fftr_axis_kernel<T, LOGL, false>, smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, fftr_axis_kernel<T, LOGL, false>, in, out, outer_ll, inner_ll,
                              Nt, P, LS, pad_mode, twiddle, deconv);
}

template <typename T, int LOGL>
cudaError_t launch_fixed(const typename Cplx<T>::type *in, typename Cplx<T>::type *out,
                         int64_t outer, int64_t inner, int Nt, int pad_mode, int sign,
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
    // lines of 16 ... 8192 points (FP32) or 16 ... 4096 points (FP64): radix-8 in registers
    if constexpr (LOGL >= 4 && LOGL <= (sizeof(T) == 4 ? 13 : 12)) {
        return launch_fftr<T, LOGL>(in, out, outer, inner, Nt, pad_mode, sign, twiddle, deconv,
                                    stream);
    }
    if (pad_mode == 2) return cudaErrorInvalidValue;  // plain lines only through the kernel above
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
                            int64_t outer, int64_t inner, int L, int Nt, int pad_mode, int sign,
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

// ------------------------------------------------------------------ fused batches
// One pass of the pruned FFT for every plan of a batch in one launch: the CTAs walk a work list
// of (plan, block) items, a block being P = kFusedFftThreads * 8 / L lines of the plan's length
// L, so every item keeps the whole CTA busy whatever L is.
namespace {

// (three CTAs per SM: at 40 registers a thread the latency-bound passes keep more lines in
// flight; measured 10% faster than two CTAs at 64 registers on the batched workload)
template <typename T, bool INV>
__global__ void __launch_bounds__(kFusedFftThreads, 3)
    fft_fused_kernel(const FusedFftPass *__restrict__ passes,
                     const FusedItem *__restrict__ items, int nitems,
                     const __grid_constant__ FusedPtrs ptrs)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *S = reinterpret_cast<C *>(smem_raw);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const FusedItem w = items[it];
        const FusedFftPass q = passes[w.plan];
        const C *in = static_cast<const C *>(q.in ? q.in : ptrs.in[w.plan]);
        C *out = static_cast<C *>(q.out ? q.out : ptrs.out[w.plan]);
        const C *tw = static_cast<const C *>(q.tw);
        const T *dc = static_cast<const T *>(q.deconv);
        switch (q.logl) {
#define GB_FUSED_FFT(LG)                                                                          \
    case LG:                                                                                      \
        fftr_block<T, LG, INV>(in, out, q.outer, q.inner, q.Nt, q.P, q.LS, q.pad_mode, tw, dc,    \
                               (long long)w.block, S);                                            \
        break;
            GB_FUSED_FFT(4)
            GB_FUSED_FFT(5)
            GB_FUSED_FFT(6)
            GB_FUSED_FFT(7)
            GB_FUSED_FFT(8)
            GB_FUSED_FFT(9)
            GB_FUSED_FFT(10)
            GB_FUSED_FFT(11)
            GB_FUSED_FFT(12)
#undef GB_FUSED_FFT
        default: break;
        }
        __syncthreads();  // the next item reuses the line buffers
    }
}

}  // namespace

template <typename T>
cudaError_t launch_fft_fused(const FusedFftPass *passes, const FusedItem *items, int nitems,
                             int sign, size_t smem, const FusedPtrs &ptrs, cudaStream_t stream)
{
    if (nitems <= 0) return cudaSuccess;
    const void *k = sign > 0 ? reinterpret_cast<const void *>(fft_fused_kernel<T, true>)
                             : reinterpret_cast<const void *>(fft_fused_kernel<T, false>);
    cudaError_t e = ensure_dynamic_smem_ptr(k, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = sign > 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                       &per_sm, fft_fused_kernel<T, true>, kFusedFftThreads, smem)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                       &per_sm, fft_fused_kernel<T, false>, kFusedFftThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidValue;
    const int blocks = std::min(nitems, per_sm * num_sms());
    if (sign > 0)
        fft_fused_kernel<T, true><<<blocks, kFusedFftThreads, smem, stream>>>(passes, items,
                                                                             nitems, ptrs);
    else
        fft_fused_kernel<T, false><<<blocks, kFusedFftThreads, smem, stream>>>(passes, items,
                                                                              nitems, ptrs);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ any even length: Bluestein
// A line of length L that is not a power of two is transformed through the chirp identity
// jk = (j^2 + k^2 - (k - j)^2) / 2:
//   X_k = sum_j x_j e^(-+2 pi i jk/L) = w_k sum_j (x_j w_j) v_(k-j),
// w_j = e^(-+pi i j^2/L), v = conj(w), a linear convolution computed as a circular one of length
// M >= 2L - 1 (a power of two) with the line FFT above: the chirped line is zero-padded to M,
// transformed, multiplied by the transform of the wrapped v (divided by M, precomputed per axis
// and direction), transformed back and chirped again. Zero padding (or cropping) and the
// deconvolution factor are applied in the first (or last) step as in the power-of-two passes.
namespace {

template <typename T>
__global__ void blu_pre_kernel(const typename Cplx<T>::type *__restrict__ in,
                               typename Cplx<T>::type *__restrict__ buf, long long lines,
                               long long inner, int L, int Nt, int M, int pad_mode, int sign,
                               const T *__restrict__ deconv,
                               const typename Cplx<T>::type *__restrict__ chirp)
{
    using C = typename Cplx<T>::type;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= lines * M) return;
    const long long l = e / M;
    const int j = (int)(e - l * M);
    C y;
    y.x = (T)0;
    y.y = (T)0;
    if (j < L) {
        const long long o = l / inner, i = l - o * inner;
        const int Lin = pad_mode == 1 ? Nt : L;
        bool take = true;
        int q = j;
        if (pad_mode == 1) {
            q = j + Nt / 2;
            if (q >= L) q -= L;
            take = q < Nt;
        }
        if (take) {
            C x = in[(o * Lin + q) * inner + i];
            if (pad_mode == 1) {
                const T d = deconv[q];
                x.x *= d;
                x.y *= d;
            }
            C w = chirp[j];
            if (sign > 0) w.y = -w.y;
            y.x = x.x * w.x - x.y * w.y;
            y.y = x.x * w.y + x.y * w.x;
        }
    }
    buf[e] = y;
}

template <typename T>
__global__ void blu_mul_kernel(typename Cplx<T>::type *__restrict__ buf, long long total, int M,
                               const typename Cplx<T>::type *__restrict__ filt)
{
    using C = typename Cplx<T>::type;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const C a = buf[e], b = filt[e % M];
    C y;
    y.x = a.x * b.x - a.y * b.y;
    y.y = a.x * b.y + a.y * b.x;
    buf[e] = y;
}

template <typename T>
__global__ void blu_post_kernel(const typename Cplx<T>::type *__restrict__ buf,
                                typename Cplx<T>::type *__restrict__ out, long long lines,
                                long long inner, int L, int Nt, int M, int pad_mode, int sign,
                                const T *__restrict__ deconv,
                                const typename Cplx<T>::type *__restrict__ chirp)
{
    using C = typename Cplx<T>::type;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= lines * L) return;
    const long long l = e / L;
    const int k = (int)(e - l * L);
    const long long o = l / inner, i = l - o * inner;
    const C a = buf[l * M + k];
    C w = chirp[k];
    if (sign > 0) w.y = -w.y;
    C y;
    y.x = a.x * w.x - a.y * w.y;
    y.y = a.x * w.y + a.y * w.x;
    if (pad_mode == 0) {  // crop to the centred I_N and deconvolve
        int q = k + Nt / 2;
        if (q >= L) q -= L;
        if (q >= Nt) return;
        const T d = deconv[q];
        y.x *= d;
        y.y *= d;
        out[(o * Nt + q) * inner + i] = y;
    } else {
        out[(o * L + k) * inner + i] = y;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_fft_axis_bluestein(const typename Cplx<T>::type *in,
                                      typename Cplx<T>::type *out, int64_t outer, int64_t inner,
                                      int L, int Nt, int pad_mode, int sign, const T *deconv,
                                      const BluesteinAxis<T> &ax, cudaStream_t stream)
{
    using C = typename Cplx<T>::type;
    if (outer <= 0 || inner <= 0) return cudaSuccess;
    const int M = ax.M;
    const long long lines = (long long)outer * inner;
    C *b0 = static_cast<C *>(ax.buf0);
    C *b1 = static_cast<C *>(ax.buf1);
    const C *chirp = static_cast<const C *>(ax.chirp);
    const C *twM = static_cast<const C *>(ax.twM);
    const C *filt = static_cast<const C *>(sign < 0 ? ax.filt_fwd : ax.filt_inv);
    const int threads = 256;
    long long total = lines * M;
    blu_pre_kernel<T><<<(unsigned)((total + threads - 1) / threads), threads, 0, stream>>>(
        in, b0, lines, inner, L, Nt, M, pad_mode, sign, deconv, chirp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_fft_axis<T>(b0, b1, lines, 1, M, M, 2, -1, twM, nullptr, stream);
    if (e != cudaSuccess) return e;
    blu_mul_kernel<T><<<(unsigned)((total + threads - 1) / threads), threads, 0, stream>>>(
        b1, total, M, filt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_fft_axis<T>(b1, b0, lines, 1, M, M, 2, +1, twM, nullptr, stream);
    if (e != cudaSuccess) return e;
    total = lines * L;
    blu_post_kernel<T><<<(unsigned)((total + threads - 1) / threads), threads, 0, stream>>>(
        b0, out, lines, inner, L, Nt, M, pad_mode, sign, deconv, chirp);
    return cudaGetLastError();
}

}  // namespace gbnfft
