// A forward 1-D NFFT that allocates no device memory at all: nfft_trafo_1d_noalloc.
//
// Who needs it: code that cannot call cudaMalloc at the point where it transforms. That
// includes code whose device memory is owned by another allocator (a framework's caching pool,
// or a host application's memory budget) that forbids raw allocations, and latency-bound loops
// that cannot afford the implicit device synchronisation of cudaMalloc / cudaFree. The planned
// path (nfft_plan_create, nfft_set_nodes) allocates tables and a workspace, so those callers
// cannot use it there.
//
// This entry point needs neither a plan nor a workspace. Everything beyond the caller's inputs
// and output lives in one fixed array in device memory, g_noalloc_scratch below (288 KiB: the
// oversampled grid, the FFT twiddles and the deconvolution factors). Every GPU that loads the
// library holds that array until the process exits. Its size caps the transform at n <= 8192
// (so N <= 4096); larger sizes are refused with NFFT_ESCRATCH.
//
// The array is shared by every call and keeps the last call's contents. Each call rewrites all
// of it that it reads (tables, then the whole grid), so nothing has to start at zero. Calls that
// overlap on the GPU (different streams, or different host threads) race on the array and give
// wrong results: serialise them.
//
// Method: the same three steps as nfft_trafo (deconvolution, FFT, window interpolation), FP64,
// Kaiser-Bessel window evaluated directly from its formula, nodes processed in the caller's order
// (no sort). The device address of the array is looked up once per device and kept for the life
// of the process, so it does not survive cudaDeviceReset.
#include <cmath>
#include <mutex>

#include "gbnfft_internal.cuh"

using namespace gbnfft;

namespace {

constexpr int kNoallocMaxn = 8192;  // largest oversampled FFT length
constexpr int kNoallocMaxN = 4096;  // largest bandwidth (N < n)
constexpr double kPiNa = 3.14159265358979323846264338327950288;

// Layout of the scratch array: grid, twiddles, deconvolution factors.
constexpr size_t kGridOff = 0;
constexpr size_t kTwOff = kGridOff + sizeof(double2) * kNoallocMaxn;
constexpr size_t kDcOff = kTwOff + sizeof(double2) * kNoallocMaxn;
constexpr size_t kScratchBytes = kDcOff + sizeof(double) * kNoallocMaxN;  // 288 KiB

// The fixed scratch. In host code this name is only a stand-in for the device symbol: host code
// must use the address from cudaGetSymbolAddress (see scratch_address), never the name itself.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch on the current device, looked up once per device (with
// that device current) and kept for the life of the process.
int scratch_address(int dev, unsigned char **out)
{
    static std::mutex mu;
    static unsigned char *addr[64] = {nullptr};
    if (dev < 0 || dev >= 64) return NFFT_EINVAL;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return NFFT_ECUDA;
        }
        addr[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = addr[dev];
    return NFFT_OK;
}

// I0 by its power series sum (z^2/4)^j / (j!)^2.
__device__ double na_bessel_i0(double z)
{
    const double q = 0.25 * z * z;
    double term = 1.0, sum = 1.0;
    for (int j = 1; j < 500; j++) {
        term *= q / ((double)j * (double)j);
        sum += term;
        if (term <= 1e-17 * sum) break;
    }
    return sum;
}

// Twiddles e^{-2 pi i j / n} and the deconvolution factors psi(0) / (n phihat(k)) of the
// normalised window (psibar = psi / psi(0)), k = i - N/2.
__global__ void noalloc_tables_kernel(double2 *tw, double *dc, int N, int n, int m, double b,
                                      double psi0)
{
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        double s, c;
        sincospi(-2.0 * (double)j / (double)n, &s, &c);
        tw[j] = make_double2(c, s);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const double w = 2.0 * kPiNa * (double)(i - N / 2) / (double)n;
        dc[i] = psi0 / na_bessel_i0((double)m * sqrt(b * b - w * w));
    }
}

// Step B for nodes in the caller's order: f_j = sum over the closed support of
// g_{l mod n} psibar(n x_j - l), psibar(t) = kscale sinh(b u) / u, u = sqrt(m^2 - t^2).
// A node that is not finite (or too large for an exact offset) gets NaN.
__global__ void noalloc_interp_kernel(const double2 *__restrict__ grid, const double *__restrict__ x,
                                      int M, int n, int m, double b, double kscale,
                                      double2 *__restrict__ f)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const double t = (double)n * x[j];
    if (!(fabs(t) < 4503599627370496.0)) {
        f[j] = make_double2(nan(""), nan(""));
        return;
    }
    const double bf = floor(t);
    const double frac = t - bf;
    const long long base = (long long)bf;
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i <= 2 * m; i++) {
        const double s = ((double)i - frac) * ((double)(2 * m - i) + frac);  // m^2 - (n x - l)^2
        double w;
        if (s > 0.0) {
            const double u = sqrt(s);
            w = kscale * sinh(b * u) / u;
        } else {
            w = s == 0.0 ? kscale * b : 0.0;
        }
        const double2 v = grid[(int)((base - m + i) & (long long)(n - 1))];
        acc.x += v.x * w;
        acc.y += v.y * w;
    }
    f[j] = acc;
}

bool aligned_to(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" int nfft_trafo_1d_noalloc(int64_t N, int64_t M, const int64_t *n_opt, int m,
                                     const double *x, const void *fhat, void *f, void *stream)
{
    if (N < 2 || (N & 1) || M < 0 || M > 0x7fffffffLL) return NFFT_EINVAL;
    if (m <= 0) m = 8;
    int64_t n = 2;
    if (n_opt) {
        n = *n_opt;
    } else {
        while (n < N) n <<= 1;
        n <<= 1;  // 2^(ceil(log2 N) + 1)
    }
    if (n <= N || (n & 1) || 2 * int64_t(m) + 2 > n) return NFFT_EINVAL;
    if ((n & (n - 1)) != 0 || m > kMaxM) return NFFT_EUNSUPPORTED;
    if (n > kNoallocMaxn || N > kNoallocMaxN) return NFFT_ESCRATCH;
    if (!fhat || !aligned_to(fhat, 16)) return NFFT_EINVAL;
    if (M > 0 && (!x || !f || !aligned_to(x, 8) || !aligned_to(f, 16))) return NFFT_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NFFT_ECUDA;
    unsigned char *scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc) return rc;
    double2 *grid = reinterpret_cast<double2 *>(scratch + kGridOff);
    double2 *tw = reinterpret_cast<double2 *>(scratch + kTwOff);
    double *dc = reinterpret_cast<double *>(scratch + kDcOff);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const double sigma = double(n) / double(N);
    const double b = kPiNa * (2.0 - 1.0 / sigma);
    const double kscale = double(m) / std::sinh(b * double(m));
    const double psi0 = std::sinh(b * double(m)) / (kPiNa * double(m));

    noalloc_tables_kernel<<<8, 256, 0, s>>>(tw, dc, (int)N, (int)n, m, b, psi0);
    if (cudaGetLastError() != cudaSuccess) return NFFT_ECUDA;
    // D and F: the pruned FFT pass of the planned path, one line, reading the caller's fhat
    if (launch_fft_axis<double>(static_cast<const double2 *>(fhat), grid, 1, 1, (int)n, (int)N,
                                true, -1, tw, dc, s) != cudaSuccess)
        return NFFT_ECUDA;
    if (M > 0) {
        const int threads = 128;
        noalloc_interp_kernel<<<(unsigned)((M + threads - 1) / threads), threads, 0, s>>>(
            grid, x, (int)M, (int)n, m, b, kscale, static_cast<double2 *>(f));
        if (cudaGetLastError() != cudaSuccess) return NFFT_ECUDA;
    }
    return NFFT_OK;
}
