// One axis pass of the d-variate FFT of Algorithm "NFFT" / "adjoint NFFT" (Section 2), with the
// deconvolution D (or D^H) and the zero padding (or cropping) fused in, so that the FFT is
// pruned: a forward transform only ever transforms lines that hold nonzero data, and an adjoint
// transform only writes the |I_N| outputs it needs.
//
// A CTA loads P lines of length L (power of two) of one axis into shared memory, runs a
// Stockham autosort FFT (radix 4, one radix-2 pass when log2 L is odd) entirely in shared
// memory, and writes the lines back. Lines along the contiguous axis are rows; lines along a
// strided axis are taken P columns at a time so that global loads and stores are coalesced.
//
// The deconvolution factor of axis t is applied in the pass of axis t (the factor of
// Algorithm "NFFT" line 2, 1/(|I_n| c_k), is a product over axes), in FP64 for both precisions.
#include "gbnfft_internal.cuh"

namespace gbnfft {

namespace {

constexpr int kRegs = 16;  // complex values a thread holds during one Stockham pass

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
// multiply by sign * i  (sign = -1: -i, sign = +1: +i)
template <typename C> __device__ __forceinline__ C cmul_i(C a, int sign)
{
    C r;
    if (sign < 0) {
        r.x = a.y;
        r.y = -a.x;
    } else {
        r.x = -a.y;
        r.y = a.x;
    }
    return r;
}

// Largest CTA per precision: FP32 lines up to 16384 points use 1024 threads; FP64 lines (up to
// 8192 points) use at most 512 threads so that each thread keeps its 16 values in registers.
template <typename T> struct FftMaxThreads { static constexpr int value = 1024; };
template <> struct FftMaxThreads<double> { static constexpr int value = 512; };

template <typename T>
__global__ void __launch_bounds__(FftMaxThreads<T>::value)
    fft_axis_kernel(const typename Cplx<T>::type *__restrict__ in,
                    typename Cplx<T>::type *__restrict__ out, long long outer, long long inner,
                    int L, int Nt, int P, int pad_mode, int sign,
                    const typename Cplx<T>::type *__restrict__ tw, const double *__restrict__ deconv)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    const int pitch = L + 1;
    const int tid = threadIdx.x;
    const int T_ = blockDim.x;
    const int Lin = pad_mode ? Nt : L;
    const int Lout = pad_mode ? L : Nt;
    const int half = Nt / 2;

    // Tile of P lines: contiguous axis -> P consecutive rows; strided axis -> P consecutive
    // columns (inner indices) of one outer index.
    long long o0, i0;
    int lines;
    if (inner == 1) {
        o0 = (long long)blockIdx.x * P;
        i0 = 0;
        lines = (int)min((long long)P, outer - o0);
    } else {
        const long long tiles_per_outer = (inner + P - 1) / P;
        o0 = blockIdx.x / tiles_per_outer;
        i0 = (blockIdx.x % tiles_per_outer) * P;
        lines = (int)min((long long)P, inner - i0);
    }

    // ---- load (zero padding + deconvolution in pad mode)
    if (pad_mode) {
        for (int e = tid; e < P * pitch; e += T_) {
            C z;
            z.x = (T)0;
            z.y = (T)0;
            s[e] = z;
        }
        __syncthreads();
    }
    for (int e = tid; e < P * Lin; e += T_) {
        int c, p;
        long long src;
        if (inner == 1) {
            c = e / Lin;
            p = e - c * Lin;
            src = (o0 + c) * Lin + p;
        } else {
            p = e / P;
            c = e - p * P;
            src = (o0 * Lin + p) * inner + i0 + c;
        }
        if (c >= lines) continue;
        C v = in[src];
        int pos = p;
        if (pad_mode) {
            const double w = deconv[p];
            v.x = (T)((double)v.x * w);
            v.y = (T)((double)v.y * w);
            pos = p - half;
            if (pos < 0) pos += L;
        }
        s[c * pitch + pos] = v;
    }
    __syncthreads();

    // ---- Stockham passes in shared memory
    for (int Ns = 1; Ns < L; ) {
        const int R = ((L / Ns) % 4 == 0) ? 4 : 2;
        const int LR = L / R;
        const int nbf = P * LR;  // butterflies in this CTA
        const int per = (nbf + T_ - 1) / T_;
        C v[kRegs];
#pragma unroll
        for (int k = 0; k < kRegs / 2; k++) {
            if (k < per && (R == 4 ? k < kRegs / 4 : true)) {
                const int bfly = tid + k * T_;
                if (bfly < nbf) {
                    const int c = bfly / LR;
                    const int j = bfly - c * LR;
                    if (R == 4) {
                        if (k < kRegs / 4) {
#pragma unroll
                            for (int r = 0; r < 4; r++) v[k * 4 + r] = s[c * pitch + j + r * LR];
                        }
                    } else {
                        v[k * 2 + 0] = s[c * pitch + j];
                        v[k * 2 + 1] = s[c * pitch + j + LR];
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kRegs / 2; k++) {
            if (k < per && (R == 4 ? k < kRegs / 4 : true)) {
                const int bfly = tid + k * T_;
                if (bfly < nbf) {
                    const int c = bfly / LR;
                    const int j = bfly - c * LR;
                    const int kk = j % Ns;
                    const int stride = L / (Ns * R);  // twiddle step for this pass
                    const int idxD = (j / Ns) * Ns * R + kk;
                    if (R == 4) {
                        if (k < kRegs / 4) {
                            C a0 = v[k * 4 + 0], a1 = v[k * 4 + 1], a2 = v[k * 4 + 2],
                              a3 = v[k * 4 + 3];
                            if (kk != 0) {
                                C w1 = tw[kk * stride], w2 = tw[2 * kk * stride],
                                  w3 = tw[3 * kk * stride];
                                if (sign > 0) {
                                    w1.y = -w1.y;
                                    w2.y = -w2.y;
                                    w3.y = -w3.y;
                                }
                                a1 = cmul(a1, w1);
                                a2 = cmul(a2, w2);
                                a3 = cmul(a3, w3);
                            }
                            // radix-4 DFT with e^{sign 2 pi i r s / 4}
                            const C t0 = cadd(a0, a2), t1 = csub(a0, a2);
                            const C t2 = cadd(a1, a3), t3 = cmul_i(csub(a1, a3), sign);
                            s[c * pitch + idxD + 0 * Ns] = cadd(t0, t2);
                            s[c * pitch + idxD + 1 * Ns] = cadd(t1, t3);
                            s[c * pitch + idxD + 2 * Ns] = csub(t0, t2);
                            s[c * pitch + idxD + 3 * Ns] = csub(t1, t3);
                        }
                    } else {
                        C a0 = v[k * 2 + 0], a1 = v[k * 2 + 1];
                        if (kk != 0) {
                            C w1 = tw[kk * stride];
                            if (sign > 0) w1.y = -w1.y;
                            a1 = cmul(a1, w1);
                        }
                        s[c * pitch + idxD] = cadd(a0, a1);
                        s[c * pitch + idxD + Ns] = csub(a0, a1);
                    }
                }
            }
        }
        __syncthreads();
        Ns *= R;
    }

    // ---- store (cropping + deconvolution in crop mode)
    for (int e = tid; e < P * Lout; e += T_) {
        int c, p;
        long long dst;
        if (inner == 1) {
            c = e / Lout;
            p = e - c * Lout;
            dst = (o0 + c) * Lout + p;
        } else {
            p = e / P;
            c = e - p * P;
            dst = (o0 * Lout + p) * inner + i0 + c;
        }
        if (c >= lines) continue;
        C v;
        if (pad_mode) {
            v = s[c * pitch + p];
        } else {
            int pos = p - half;
            if (pos < 0) pos += L;
            v = s[c * pitch + pos];
            const double w = deconv[p];
            v.x = (T)((double)v.x * w);
            v.y = (T)((double)v.y * w);
        }
        out[dst] = v;
    }
}

}  // namespace

// Elements per CTA: E = P * L with P = E_target / L lines (at least one); one thread per 16
// elements, so each thread holds one radix-4 butterfly group of <= 16 values per pass.
template <typename T>
cudaError_t launch_fft_axis(const typename Cplx<T>::type *in, typename Cplx<T>::type *out,
                            int64_t outer, int64_t inner, int L, int Nt, bool pad_mode, int sign,
                            const typename Cplx<T>::type *twiddle, const double *deconv,
                            cudaStream_t stream)
{
    using C = typename Cplx<T>::type;
    if (outer <= 0 || inner <= 0) return cudaSuccess;
    const int E_target = 4096;
    int P = E_target / L;
    if (P < 1) P = 1;
    if (inner > 1 && P > inner) P = (int)inner;
    if (inner == 1 && P > outer) P = (int)outer;
    int threads = (P * L + kRegs - 1) / kRegs;
    threads = ((threads + 31) / 32) * 32;
    if (threads > FftMaxThreads<T>::value) return cudaErrorInvalidValue;
    const size_t smem = (size_t)P * (L + 1) * sizeof(C);
    long long blocks;
    if (inner == 1)
        blocks = (outer + P - 1) / P;
    else
        blocks = outer * ((inner + P - 1) / P);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = ensure_dynamic_smem(fft_axis_kernel<T>, smem);
        if (e != cudaSuccess) return e;
    }
    fft_axis_kernel<T><<<(unsigned)blocks, threads, smem, stream>>>(
        in, out, outer, inner, L, Nt, P, pad_mode ? 1 : 0, sign, twiddle, deconv);
    return cudaGetLastError();
}

template cudaError_t launch_fft_axis<float>(const float2 *, float2 *, int64_t, int64_t, int, int,
                                            bool, int, const float2 *, const double *,
                                            cudaStream_t);
template cudaError_t launch_fft_axis<double>(const double2 *, double2 *, int64_t, int64_t, int,
                                             int, bool, int, const double2 *, const double *,
                                             cudaStream_t);

}  // namespace gbnfft
