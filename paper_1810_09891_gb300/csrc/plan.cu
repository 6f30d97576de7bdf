// C ABI of gbnfft (declared in include/gbnfft.h): plan creation and validation, host-side
// tables (deconvolution factors and FFT twiddles, both in FP64), workspace layout, and the
// orchestration of the kernels for set_nodes, the forward NFFT (Algorithm "NFFT": D, F, B),
// the adjoint NFFT (Algorithm "adjoint NFFT": B^H, F^H, D^H) and the node gradient.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gbnfft_internal.cuh"

using namespace gbnfft;

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int ilog2(int64_t v)
{
    int r = 0;
    while ((int64_t(1) << r) < v) r++;
    return r;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Modified Bessel function I0 by its power series sum (z^2/4)^j / (j!)^2 (terms all positive).
double bessel_i0(double z)
{
    const double q = 0.25 * z * z;
    double term = 1.0, sum = 1.0;
    for (int j = 1; j < 1000; j++) {
        term *= q / (double(j) * double(j));
        sum += term;
        if (term <= 1e-17 * sum) break;
    }
    return sum;
}

// e^{-2 pi i j / L} with the angle reduced to the first octant (exact symmetry) before calling
// cos / sin, so that the table is correctly rounded up to the host libm's accuracy.
void twiddle(int64_t j, int64_t L, double *re, double *im)
{
    j %= L;
    const int64_t q = (4 * j) / L;          // quadrant
    const int64_t r = 4 * j - q * L;        // angle inside the quadrant, in units of (pi/2)/L
    double cr, sr;
    if (2 * r <= L) {
        const double th = 0.5 * kPi * double(r) / double(L);
        cr = std::cos(th);
        sr = std::sin(th);
    } else {
        const double th = 0.5 * kPi * double(L - r) / double(L);
        cr = std::sin(th);
        sr = std::cos(th);
    }
    double c, s;  // rotate (cr, sr) by q quarter turns
    switch (q & 3) {
    case 0: c = cr; s = sr; break;
    case 1: c = -sr; s = cr; break;
    case 2: c = -cr; s = -sr; break;
    default: c = sr; s = -cr; break;
    }
    *re = c;
    *im = -s;
}

// ------------------------------------------------------------------------------ windows
// The window pairs (psi in grid units t = n x, and n * phihat(k), the Fourier transform of the
// untruncated window at frequency k / n). Kaiser-Bessel is the paper's default (Section 4.1);
// Gaussian, B-spline and sinc are the alternatives it names there, with their standard pairs.
enum WindowKind { kWinKB = 0, kWinGauss = 1, kWinBspline = 2, kWinSinc = 3 };

// Shape parameter: KB b = pi (2 - 1/sigma); Gaussian b = 2 sigma m / ((2 sigma - 1) pi);
// sinc a = (2 sigma - 1) / (2 m sigma); B-spline none.
double window_param(int kind, double sigma, int m)
{
    switch (kind) {
    case kWinGauss: return 2.0 * sigma * m / ((2.0 * sigma - 1.0) * kPi);
    case kWinSinc: return (2.0 * sigma - 1.0) / (2.0 * m * sigma);
    case kWinBspline: return 0.0;
    default: return kPi * (2.0 - 1.0 / sigma);
    }
}

// Centred cardinal B-spline M_p(t) by the order recursion, evaluated bottom-up over the
// p (p+1)/2 shifted points it needs (values non-negative, no cancellation).
double cardinal_bspline(int p, double t)
{
    if (!(t > -0.5 * p && t < 0.5 * p)) return 0.0;
    double v[40];
    for (int j = 0; j < p; j++) {  // level 1 at u_j = t + (p - 1)/2 - j
        const double u = t + 0.5 * (p - 1) - j;
        v[j] = (u >= -0.5 && u < 0.5) ? 1.0 : 0.0;
    }
    for (int k = 2; k <= p; k++) {  // level k at u_j = t + (p - k)/2 - j, j = 0..p-k
        for (int j = 0; j <= p - k; j++) {
            const double u = t + 0.5 * (p - k) - j;
            v[j] = ((0.5 * k + u) * v[j] + (0.5 * k - u) * v[j + 1]) / (k - 1);
        }
    }
    return v[0];
}

double sinc_host(double u) { return u == 0.0 ? 1.0 : std::sin(u) / u; }

// Truncated window psi(t), |t| <= m.
double psi_host(int kind, double t, int m, double prm)
{
    if (std::fabs(t) > double(m)) return 0.0;
    switch (kind) {
    case kWinGauss: return std::exp(-t * t / prm);
    case kWinBspline: return cardinal_bspline(2 * m, t);
    case kWinSinc: return std::pow(sinc_host(kPi * prm * t), 2 * m);
    default: {
        const double s = (double(m) - t) * (double(m) + t);
        if (s <= 0.0) return prm / kPi;
        const double u = std::sqrt(s);
        return std::sinh(prm * u) / (kPi * u);
    }
    }
}

// n * phihat(k): the Fourier transform of the untruncated psi at frequency k / n.
double nphihat_host(int kind, double k, double n, int m, double prm)
{
    const double nu = k / n;
    switch (kind) {
    case kWinGauss: return std::sqrt(kPi * prm) * std::exp(-prm * kPi * kPi * nu * nu);
    case kWinBspline: return std::pow(sinc_host(kPi * nu), 2 * m);
    case kWinSinc: return cardinal_bspline(2 * m, nu / prm) / prm;
    default: {
        const double w = 2.0 * kPi * nu;
        return bessel_i0(double(m) * std::sqrt(prm * prm - w * w));
    }
    }
}

// d psi / d t at t = m (from inside the support).
double dpsi_edge_host(int kind, int m, double prm)
{
    switch (kind) {
    case kWinGauss: return -2.0 * m / prm * std::exp(-double(m) * m / prm);
    case kWinBspline: return 0.0;  // M_{2m} is flat (C^{2m-2}) at its support edge
    case kWinSinc: {
        const double u = kPi * prm * m;
        const double ds = (u * std::cos(u) - std::sin(u)) / (u * u);
        return 2.0 * m * std::pow(sinc_host(u), 2 * m - 1) * ds * kPi * prm;
    }
    default: return -double(m) * prm * prm * prm / (3.0 * kPi);
    }
}

// Monomial coefficients (in z = 2 frac - 1) of the degree-deg Chebyshev interpolant of
// frac -> psibar(frac + m - i) = psi(frac + m - i) / psi(0) on [0, 1] (interpolation at the
// deg + 1 Chebyshev points).
void fit_tap_poly(int kind, int m, double prm, int i, int deg, double *mono)
{
    const int n = deg + 1;
    const double psi0 = psi_host(kind, 0.0, m, prm);
    double f[32], c[32], Tprev[32], Tcur[32], Tnext[32];
    for (int k = 0; k < n; k++) {
        const double z = std::cos(kPi * (k + 0.5) / n);
        f[k] = psi_host(kind, 0.5 * (z + 1.0) + double(m) - double(i), m, prm) / psi0;
    }
    for (int j = 0; j < n; j++) {
        double acc = 0.0;
        for (int k = 0; k < n; k++) acc += f[k] * std::cos(kPi * j * (k + 0.5) / n);
        c[j] = 2.0 * acc / n;
    }
    c[0] *= 0.5;
    for (int k = 0; k < n; k++) mono[k] = Tprev[k] = Tcur[k] = 0.0;
    Tprev[0] = 1.0;  // T_0
    Tcur[1] = 1.0;   // T_1
    mono[0] = c[0];
    if (n > 1) mono[1] += c[1];
    for (int j = 2; j < n; j++) {
        for (int k = 0; k < n; k++) Tnext[k] = (k > 0 ? 2.0 * Tcur[k - 1] : 0.0) - Tprev[k];
        for (int k = 0; k < n; k++) {
            mono[k] += c[j] * Tnext[k];
            Tprev[k] = Tcur[k];
            Tcur[k] = Tnext[k];
        }
    }
}

struct Region {
    size_t off = 0, bytes = 0;
};

// Every device allocation of the library goes through here. Failure injection for tests (host
// side only, nothing reaches the GPU): when the environment variable GBNFFT_FAIL_ALLOC names this
// allocation's site ("tables", "workspace", "stage", "lin"; a comma-separated list, or "all"),
// the allocation is refused as if the device were out of memory.
bool alloc_refused(const char *site)
{
    const char *v = std::getenv("GBNFFT_FAIL_ALLOC");
    if (!v || !*v) return false;
    if (std::strcmp(v, "all") == 0) return true;
    const size_t n = std::strlen(site);
    for (const char *q = v; *q;) {
        const char *e = std::strchr(q, ',');
        const size_t len = e ? size_t(e - q) : std::strlen(q);
        if (len == n && std::strncmp(q, site, n) == 0) return true;
        if (!e) break;
        q = e + 1;
    }
    return false;
}

cudaError_t dev_alloc(void **ptr, size_t bytes, const char *site)
{
    *ptr = nullptr;
    if (alloc_refused(site)) return cudaErrorMemoryAllocation;
    return cudaMalloc(ptr, bytes);
}

}  // namespace

struct gbnfft_plan {
    int device = 0;
    int d = 0, m = 0, dtype = 0;
    int64_t N[3] = {0, 0, 0}, n[3] = {0, 0, 0}, M = 0;
    Geom geom{};
    cudaStream_t stream = nullptr;
    size_t csize = 0;  // bytes per complex value
    size_t rsize = 0;  // bytes per real value
    int64_t G = 0;     // |I_n|
    int64_t NN = 0;    // |I_N|
    int64_t Bsz = 0;   // complex values of the second FFT buffer
    int nbins = 0;
    int max_subs = 0;
    int64_t bin_req[3] = {0, 0, 0};  // requested bin sizes (0 = default)
    int64_t sub_req = 0;             // requested nodes per spreading subproblem (0 = default)
    int sub_max = kMaxSub;
    int window = 0;  // WindowKind
    int lin_k = 0;            // PRE_LIN_PSI: samples per unit of t of the window tables, 0 = off
    void *lin_tab = nullptr;  // device tables (plan precision), d x (K + 1) x 2m values
    // plan-owned device tables: [deconv_t, twiddles_t]_t, window polynomials, status word
    void *tables = nullptr;
    size_t off_dc[3] = {0, 0, 0}, off_tw[3] = {0, 0, 0}, off_poly = 0, off_status = 0;
    size_t tbytes = 0;
    std::vector<unsigned char> poly_host;  // host copy of the window polynomials
    // axes whose FFT length is not a power of two (Bluestein): convolution length and tables
    int blu_M[3] = {0, 0, 0};
    size_t off_chirp[3] = {0, 0, 0}, off_ff[3] = {0, 0, 0}, off_fi[3] = {0, 0, 0};
    size_t off_twM[3] = {0, 0, 0};
    size_t blu_elems = 0;  // values per Bluestein scratch buffer (max over axes of lines x M)
    void *deconv[3] = {nullptr, nullptr, nullptr};  // plan precision
    void *tw[3] = {nullptr, nullptr, nullptr};
    int *d_status = nullptr;
    // workspace
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    // gA, gB: grid and pruned intermediate of the adjoint; gC, gD: those of the forward
    // transform and the node gradient (separate, so that a forward and an adjoint of one plan
    // may run at the same time on different streams)
    Region gA, gB, gC, gD, rec, perm, binrank, bincount, binstart, substart, nsub, subs, blu;
    Region rowcount, rowstart;  // row sub-bins of the bins: node counts and first positions
    // stripe-form spreading work (d = 2): super-bin counts, scans and items
    Region sbcount, sbstart, sbsub, sbn, sitems;
    int stripe_R = 0, stripe_nsb1 = 0, stripe_nsb = 0, stripe_max_items = 0;
    int64_t stripe_item_req = 0;  // requested nodes per stripe work item (0 = default)
    size_t ws_need = 0;
    bool nodes_ready = false;
    bool stripe_ready = false;  // stripe-form work items built for the current node set
    // host-call staging (plan-owned)
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // per-stage CUDA-event timing (nfft_profile)
    struct ProfPair {
        cudaEvent_t a, b;
        int stage;
    };
    bool prof_on = false;
    std::vector<ProfPair> prof;
    size_t prof_used = 0;
};

namespace {

int cuda_fail(cudaError_t e)
{
    if (e == cudaErrorMemoryAllocation) return NFFT_ENOMEM;
    return e == cudaSuccess ? NFFT_OK : NFFT_ECUDA;
}

#define GB_CHECK(expr)                                                                            \
    do {                                                                                          \
        cudaError_t _e = (expr);                                                                  \
        if (_e != cudaSuccess) return cuda_fail(_e);                                              \
    } while (0)

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

void layout_workspace(gbnfft_plan *p)
{
    size_t off = 0;
    auto put = [&](Region &r, size_t bytes) {
        off = align_up(off, 256);
        r.off = off;
        r.bytes = bytes;
        off += bytes;
    };
    const size_t recsz = p->dtype == NFFT_FP32 ? sizeof(RecF) : sizeof(RecD);
    put(p->gA, size_t(p->G) * p->csize);
    put(p->gB, size_t(p->Bsz) * p->csize);
    put(p->gC, size_t(p->G) * p->csize);
    put(p->gD, size_t(p->Bsz) * p->csize);
    put(p->rec, size_t(p->M) * recsz);
    put(p->perm, size_t(p->M) * sizeof(int));
    put(p->binrank, size_t(p->M) * sizeof(int2));
    put(p->bincount, size_t(p->nbins) * sizeof(int));
    put(p->binstart, size_t(p->nbins) * sizeof(int));
    put(p->substart, size_t(p->nbins) * sizeof(int));
    const size_t S0 = size_t(p->geom.bs[0]) * (p->d == 3 ? p->geom.bs[1] : 1);
    put(p->rowcount, size_t(p->nbins) * S0 * sizeof(int));
    put(p->rowstart, size_t(p->nbins) * S0 * sizeof(int));
    put(p->nsub, 16);
    put(p->subs, size_t(p->max_subs) * sizeof(SubProb));
    put(p->blu, 2 * p->blu_elems * p->csize);
    put(p->sbcount, size_t(p->stripe_nsb) * sizeof(int));
    put(p->sbstart, size_t(p->stripe_nsb) * sizeof(int));
    put(p->sbsub, size_t(p->stripe_nsb) * sizeof(int));
    put(p->sbn, 16);
    put(p->sitems, size_t(p->stripe_max_items) * sizeof(SubProb));
    p->ws_need = align_up(off, 256);
}

// Bin (tile) sizes per axis: the requested ones, else the defaults (1-D 1024; 2-D 4 x 8 in FP32
// with m <= 4, whose tiles the rows spreading form holds a half-warp per tile, else 8 x 16; 3-D
// 8 x 8 x 16), clipped to n_t; nodes per spreading work item: the requested number, else for
// 2-D FP32 64 (bins of at most 32 cells) or 128, and 1024 otherwise (the fastest choices
// measured with the default spreading forms on a radial trajectory, whose bins hold very
// different node counts). Recomputes the bin
// counts and the workspace layout.
void setup_bins(gbnfft_plan *p)
{
    Geom &g = p->geom;
    const int64_t bin_default[3][3] = {{1024, 0, 0}, {8, 16, 0}, {8, 8, 16}};
    int64_t nbins = 1;
    for (int t = 0; t < kMaxDim; t++) {
        if (t >= p->d) {
            g.bs[t] = 1;
            g.bslog[t] = 0;
            g.nb[t] = 1;
            continue;
        }
        int64_t bs = p->bin_req[t] > 0 ? p->bin_req[t] : bin_default[p->d - 1][t];
        // FP32 2-D with m <= 4: 4 x 8 bins, whose tiles (at most 16 cells wide) the rows
        // spreading form holds a half-warp per tile
        if (p->bin_req[t] <= 0 && p->d == 2 && p->dtype == NFFT_FP32 && p->m <= 4)
            bs = t == 0 ? 4 : 8;
        if (is_pow2(p->n[t])) {
            if (bs > p->n[t]) bs = p->n[t];  // one bin covers the axis
        } else {
            int64_t cap = 1;  // the largest power of two <= n/2 (the last bin may be partial)
            while (cap * 2 <= p->n[t] / 2) cap *= 2;
            if (bs > cap) bs = cap;
        }
        g.bs[t] = (int)bs;
    }
    // default bins shrink (largest first) until one tile with its 2m halo fits in shared memory
    // beside the window tables (large m in FP64 3-D)
    const size_t tile_limit = 200 * 1024;
    for (;;) {
        size_t cells = 1;
        int big = -1;
        for (int t = 0; t < p->d; t++) {
            cells *= size_t(g.bs[t] + 2 * p->m);
            if (p->bin_req[t] <= 0 && g.bs[t] > 1 && (big < 0 || g.bs[t] > g.bs[big])) big = t;
        }
        if (cells * p->csize <= tile_limit || big < 0) break;
        g.bs[big] /= 2;
    }
    for (int t = 0; t < kMaxDim; t++) {
        if (t >= p->d) continue;
        g.bslog[t] = ilog2(g.bs[t]);
        g.nb[t] = (int)((p->n[t] + g.bs[t] - 1) / g.bs[t]);
        nbins *= g.nb[t];
    }
    p->nbins = (int)nbins;
    // 2-D FP32: short subproblems even out the load of the heavy bins (64 nodes for the rows
    // form's 4 x 8 bins, 128 for larger bins)
    p->sub_max = p->sub_req > 0 ? (int)p->sub_req
                                : (p->d == 2 && p->dtype == NFFT_FP32
                                       ? (g.bs[0] * g.bs[1] <= 32 ? 64 : 128)
                                       : kMaxSub);
    p->max_subs = (int)(nbins + (p->M + p->sub_max - 1) / p->sub_max + 1);
    // stripe-form work (d = 2): stripes of stripe_width(m) >= 2m cells made of whole sort bins,
    // kStripeS stripes per super-bin; the super-bin tile must not wrap onto itself
    p->stripe_R = p->stripe_nsb1 = p->stripe_nsb = p->stripe_max_items = 0;
    if (p->d == 2) {
        const int W = stripe_width(p->m);
        const int span = kStripeS * W;
        if (g.bs[1] <= W && span + 2 * p->m <= p->n[1]) {
            p->stripe_R = W / g.bs[1];
            const int bins_per_sb = kStripeS * p->stripe_R;
            p->stripe_nsb1 = (g.nb[1] + bins_per_sb - 1) / bins_per_sb;
            p->stripe_nsb = g.nb[0] * p->stripe_nsb1;
            const int64_t item = p->stripe_item_req > 0 ? p->stripe_item_req : kStripeItemDefault;
            p->stripe_max_items = (int)(p->stripe_nsb + (p->M + item - 1) / item + 1);
        }
    }
    layout_workspace(p);
}

template <typename R> R *at(gbnfft_plan *p, const Region &r)
{
    return reinterpret_cast<R *>(p->ws + r.off);
}

int ensure_workspace(gbnfft_plan *p)
{
    if (p->ws) return NFFT_OK;
    void *ptr = nullptr;
    cudaError_t e = dev_alloc(&ptr, p->ws_need, "workspace");
    if (e != cudaSuccess) {
        cudaGetLastError();
        return NFFT_ENOMEM;
    }
    p->ws = static_cast<char *>(ptr);
    p->ws_bytes = p->ws_need;
    p->ws_owned = true;
    return NFFT_OK;
}

// Stage timing: a pair of events recorded on the plan's stream around one stage.
int prof_begin(gbnfft_plan *p, int stage)
{
    if (!p->prof_on) return -1;
    if (p->prof_used == p->prof.size()) {
        gbnfft_plan::ProfPair pp{};
        if (cudaEventCreate(&pp.a) != cudaSuccess) return -1;
        if (cudaEventCreate(&pp.b) != cudaSuccess) {
            cudaEventDestroy(pp.a);
            return -1;
        }
        p->prof.push_back(pp);
    }
    const int idx = (int)p->prof_used++;
    p->prof[idx].stage = stage;
    cudaEventRecord(p->prof[idx].a, p->stream);
    return idx;
}

void prof_end(gbnfft_plan *p, int idx)
{
    if (idx >= 0) cudaEventRecord(p->prof[idx].b, p->stream);
}

// Names of the stages for NVTX ranges (one range per stage and call, on the calling thread;
// a profiler that records NVTX shows them around the stage's launches).
const char *const kStageName[NFFT_NUM_STAGES] = {
    "gbnfft set_nodes", "gbnfft fft_forward", "gbnfft interp", "gbnfft zero_grid",
    "gbnfft spread",    "gbnfft fft_adjoint", "gbnfft grad"};

struct ProfScope {
    gbnfft_plan *p;
    int idx;
    ProfScope(gbnfft_plan *pp, int stage) : p(pp), idx(prof_begin(pp, stage))
    {
        nvtxRangePushA(kStageName[stage]);
    }
    ~ProfScope()
    {
        prof_end(p, idx);
        nvtxRangePop();
    }
};

// One axis pass of the oversampled FFT along axis t: the power-of-two kernels, or Bluestein
// through the axis' tables and the workspace scratch.
template <typename T>
cudaError_t fft_pass(gbnfft_plan *p, int t, const typename Cplx<T>::type *in,
                     typename Cplx<T>::type *out, int64_t outer, int64_t inner, bool pad, int sign)
{
    using C = typename Cplx<T>::type;
    const T *dc = static_cast<const T *>(p->deconv[t]);
    if (!p->blu_M[t])
        return launch_fft_axis<T>(in, out, outer, inner, (int)p->n[t], (int)p->N[t], pad ? 1 : 0,
                                  sign, static_cast<const C *>(p->tw[t]), dc, p->stream);
    char *tb = static_cast<char *>(p->tables);
    BluesteinAxis<T> ax;
    ax.M = p->blu_M[t];
    ax.chirp = tb + p->off_chirp[t];
    ax.filt_fwd = tb + p->off_ff[t];
    ax.filt_inv = tb + p->off_fi[t];
    ax.twM = tb + p->off_twM[t];
    ax.buf0 = p->ws + p->blu.off;
    ax.buf1 = p->ws + p->blu.off + p->blu_elems * p->csize;
    return launch_fft_axis_bluestein<T>(in, out, outer, inner, (int)p->n[t], (int)p->N[t],
                                        pad ? 1 : 0, sign, dc, ax, p->stream);
}

// Forward FFT passes with D fused: fhat (centred, |I_N|) -> gC (|I_n|, natural order), through
// gD.
template <typename T> int forward_grid(gbnfft_plan *p, const void *fhat)
{
    using C = typename Cplx<T>::type;
    const C *in = static_cast<const C *>(fhat);
    C *A = at<C>(p, p->gC), *B = at<C>(p, p->gD);
    const int64_t *N = p->N, *n = p->n;
    if (p->d == 1) {
        GB_CHECK(fft_pass<T>(p, 0, in, A, 1, 1, true, -1));
    } else if (p->d == 2) {
        GB_CHECK(fft_pass<T>(p, 1, in, B, N[0], 1, true, -1));
        GB_CHECK(fft_pass<T>(p, 0, B, A, 1, n[1], true, -1));
    } else {
        GB_CHECK(fft_pass<T>(p, 2, in, A, N[0] * N[1], 1, true, -1));
        GB_CHECK(fft_pass<T>(p, 1, A, B, N[0], n[2], true, -1));
        GB_CHECK(fft_pass<T>(p, 0, B, A, 1, n[1] * n[2], true, -1));
    }
    return NFFT_OK;
}

// Inverse FFT passes with D^H fused: gA (|I_n|) -> fhat (|I_N|). gA is overwritten.
template <typename T> int adjoint_grid(gbnfft_plan *p, void *fhat)
{
    using C = typename Cplx<T>::type;
    C *out = static_cast<C *>(fhat);
    C *A = at<C>(p, p->gA), *B = at<C>(p, p->gB);
    const int64_t *N = p->N, *n = p->n;
    if (p->d == 1) {
        GB_CHECK(fft_pass<T>(p, 0, A, out, 1, 1, false, +1));
    } else if (p->d == 2) {
        GB_CHECK(fft_pass<T>(p, 0, A, B, 1, n[1], false, +1));
        GB_CHECK(fft_pass<T>(p, 1, B, out, N[0], 1, false, +1));
    } else {
        GB_CHECK(fft_pass<T>(p, 0, A, B, 1, n[1] * n[2], false, +1));
        GB_CHECK(fft_pass<T>(p, 1, B, A, N[0], n[2], false, +1));
        GB_CHECK(fft_pass<T>(p, 2, A, out, N[0] * N[1], 1, false, +1));
    }
    return NFFT_OK;
}

template <typename T> int do_set_nodes(gbnfft_plan *p, const void *x)
{
    using Rec = typename RecOf<T>::type;
    ProfScope ps(p, NFFT_STAGE_SET_NODES);
    cudaStream_t s = p->stream;
    int *count = at<int>(p, p->bincount);
    int *rows = at<int>(p, p->rowcount);
    const int S0 = p->geom.bs[0] * (p->d == 3 ? p->geom.bs[1] : 1);  // row sub-bins per bin
    GB_CHECK(cudaMemsetAsync(rows, 0, size_t(p->nbins) * S0 * sizeof(int), s));
    GB_CHECK(launch_node_bin<T>(p->geom, static_cast<const T *>(x), p->M, rows,
                                at<int2>(p, p->binrank), p->d_status, s));
    GB_CHECK(launch_bin_totals(rows, S0, p->nbins, count, s));
    // 2-D: bins in 2 x 2 blocks (B then walks compact regions of twice the bin size); not when
    // stripes of more than two bins need their bins' nodes contiguous
    const bool blocked = p->d == 2 && p->stripe_R <= 2;
    GB_CHECK(launch_bin_scan(count, at<int>(p, p->binstart), at<int>(p, p->substart),
                             at<int>(p, p->nsub), p->nbins, p->sub_max, s,
                             blocked ? p->geom.nb[0] : 0, blocked ? p->geom.nb[1] : 0));
    GB_CHECK(launch_sub_starts(rows, at<int>(p, p->binstart), S0, p->nbins,
                               at<int>(p, p->rowstart), s));
    GB_CHECK(launch_node_scatter<T>(p->geom, static_cast<const T *>(x), p->M,
                                    at<int2>(p, p->binrank), at<int>(p, p->rowstart),
                                    at<Rec>(p, p->rec), at<int>(p, p->perm), s));
    GB_CHECK(launch_fill_subprobs(count, at<int>(p, p->binstart), at<int>(p, p->substart),
                                  at<SubProb>(p, p->subs), p->nbins, p->sub_max, s));
    p->stripe_ready = false;  // the stripe form's work items are built when it first runs
    return NFFT_OK;
}

// The stripe form's work items for the current node set (on the plan's stream, once per
// set_nodes, on the first adjoint that uses the form).
cudaError_t stripe_items(gbnfft_plan *p)
{
    if (p->stripe_R <= 0 || p->stripe_ready) return cudaSuccess;
    const int item = p->stripe_item_req > 0 ? (int)p->stripe_item_req : kStripeItemDefault;
    const cudaError_t e = launch_stripe_items(
        at<int>(p, p->bincount), p->geom.nb[0], p->geom.nb[1], p->stripe_R, p->stripe_nsb1,
        at<int>(p, p->sbcount), at<int>(p, p->sbstart), at<int>(p, p->sbsub), at<int>(p, p->sbn),
        at<SubProb>(p, p->sitems), item, p->stream);
    if (e == cudaSuccess) p->stripe_ready = true;
    return e;
}

// The plan's geometry with the stripe-form work of the current node set attached.
Geom spread_geom(gbnfft_plan *p)
{
    Geom g = p->geom;
    g.sw = StripeWork{};
    if (p->stripe_R > 0) {
        g.sw.bin_start = at<int>(p, p->binstart);
        g.sw.bin_count = at<int>(p, p->bincount);
        g.sw.items = at<SubProb>(p, p->sitems);
        g.sw.work = at<int>(p, p->sbn);
        g.sw.max_items = p->stripe_max_items;
        g.sw.R = p->stripe_R;
        g.sw.nsb1 = p->stripe_nsb1;
    }
    return g;
}

template <typename T> int do_trafo(gbnfft_plan *p, const void *fhat, void *f)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    int rc;
    {
        ProfScope ps(p, NFFT_STAGE_FFT_FORWARD);
        rc = forward_grid<T>(p, fhat);
    }
    if (rc) return rc;
    ProfScope ps(p, NFFT_STAGE_INTERP);
    GB_CHECK(launch_interp<T>(p->geom, at<C>(p, p->gC), at<Rec>(p, p->rec), at<int>(p, p->perm),
                              p->M, at<SubProb>(p, p->subs), at<int>(p, p->nsub), p->max_subs,
                              static_cast<C *>(f), p->stream));
    return NFFT_OK;
}

template <typename T> int do_adjoint(gbnfft_plan *p, const void *f, void *fhat)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    {
        ProfScope ps(p, NFFT_STAGE_ZERO_GRID);
        GB_CHECK(cudaMemsetAsync(at<C>(p, p->gA), 0, size_t(p->G) * p->csize, p->stream));
    }
    {
        ProfScope ps(p, NFFT_STAGE_SPREAD);
        if (p->geom.spread_method == kSpreadStripe) GB_CHECK(stripe_items(p));
        GB_CHECK(launch_spread<T>(spread_geom(p), static_cast<const C *>(f), at<Rec>(p, p->rec),
                                  at<int>(p, p->perm), at<SubProb>(p, p->subs),
                                  at<int>(p, p->nsub), p->max_subs, at<C>(p, p->gA), p->stream));
    }
    ProfScope ps(p, NFFT_STAGE_FFT_ADJOINT);
    return adjoint_grid<T>(p, fhat);
}

template <typename T> int do_grad(gbnfft_plan *p, const void *coef, const void *w, void *gx)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    int rc;
    {
        ProfScope ps(p, NFFT_STAGE_FFT_FORWARD);
        rc = forward_grid<T>(p, coef);
    }
    if (rc) return rc;
    ProfScope ps(p, NFFT_STAGE_GRAD);
    GB_CHECK(launch_grad<T>(p->geom, at<C>(p, p->gC), at<Rec>(p, p->rec), at<int>(p, p->perm),
                            p->M, static_cast<const C *>(w), static_cast<T *>(gx), p->stream));
    return NFFT_OK;
}

int set_device(gbnfft_plan *p)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return NFFT_ECUDA;
    if (cur != p->device && cudaSetDevice(p->device) != cudaSuccess) return NFFT_ECUDA;
    return NFFT_OK;
}

int check_dev_ptr(const gbnfft_plan *p, const void *ptr, int64_t count)
{
    if (count == 0) return NFFT_OK;
    if (!ptr) return NFFT_EINVAL;
    if (!aligned(ptr, p->csize)) return NFFT_EINVAL;
    return NFFT_OK;
}

}  // namespace

namespace {

// In-place forward DFT X_k = sum_j x_j e^(-2 pi i jk/M) of length M = 2^k in FP64 (iterative
// radix 2), for the Bluestein filter spectra built at plan creation.
void host_fft_pow2(std::vector<std::complex<double>> &a)
{
    const int64_t M = (int64_t)a.size();
    for (int64_t i = 1, j = 0; i < M; i++) {
        int64_t bit = M >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (int64_t len = 2; len <= M; len <<= 1) {
        for (int64_t i = 0; i < M; i += len) {
            for (int64_t k = 0; k < len / 2; k++) {
                double re, im;
                twiddle(k, len, &re, &im);  // e^(-2 pi i k / len)
                const std::complex<double> w(re, im);
                const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}

template <typename CT, typename RT>
void put_complex(char *dst, int64_t i, double re, double im)
{
    CT v;
    v.x = (RT)re;
    v.y = (RT)im;
    reinterpret_cast<CT *>(dst)[i] = v;
}

}  // namespace

extern "C" {

const char *nfft_strerror(int code)
{
    switch (code) {
    case NFFT_OK: return "success";
    case NFFT_EINVAL: return "invalid argument";
    case NFFT_ENOMEM: return "out of device memory or workspace too small";
    case NFFT_ECUDA: return "CUDA runtime error";
    case NFFT_ENOTREADY: return "nodes not set (call nfft_set_nodes first)";
    case NFFT_EBADNODE: return "a node coordinate is NaN, infinite or out of range";
    case NFFT_ETIMEOUT: return "a device-side wait timed out";
    case NFFT_EUNSUPPORTED: return "parameters valid but not supported by this build";
    case NFFT_ESCRATCH: return "problem larger than the fixed scratch of the no-allocation entry point";
    default: return "unknown error";
    }
}

int nfft_use_device(int device)
{
    return cudaSetDevice(device) == cudaSuccess ? NFFT_OK : NFFT_ECUDA;
}

// Per-axis window shape parameter and the edge constants the kernels take by value:
// psibar(m) (the extra tap of a node on a grid point) and d psibar / dt at t = m.
static void set_window_constants(gbnfft_plan *p)
{
    Geom &g = p->geom;
    for (int t = 0; t < p->d; t++) {
        const double sigma = double(p->n[t]) / double(p->N[t]);
        const double prm = window_param(p->window, sigma, p->m);
        const double psi0 = psi_host(p->window, 0.0, p->m, prm);
        g.win[t].prm = prm;
        g.win[t].edge_w = psi_host(p->window, double(p->m), p->m, prm) / psi0;
        g.win[t].edge_dw = dpsi_edge_host(p->window, p->m, prm) / psi0;
        if (p->lin_k > 0) {  // slope of the last table segment inside the support
            const double K = double(p->lin_k);
            g.win[t].edge_dw =
                (g.win[t].edge_w - psi_host(p->window, double(p->m) - 1.0 / K, p->m, prm) / psi0) *
                K;
        }
    }
}

// PRE_LIN_PSI tables for the plan's window: lt[j * 2m + i - 1] = psibar(j / K + m - i) per axis,
// uploaded to a plan-owned allocation (replaced when K or the window changes).
static int build_lin_tables(gbnfft_plan *p)
{
    Geom &g = p->geom;
    if (p->lin_tab) {
        cudaDeviceSynchronize();
        cudaFree(p->lin_tab);
        p->lin_tab = nullptr;
    }
    g.lin = nullptr;
    g.lin_k = 0;
    if (p->lin_k <= 0) return NFFT_OK;
    const int K = p->lin_k, m = p->m, W = 2 * m;
    const size_t per_axis = size_t(K + 1) * W;
    std::vector<double> h(per_axis * p->d);
    for (int t = 0; t < p->d; t++) {
        const double prm = g.win[t].prm;
        const double psi0 = psi_host(p->window, 0.0, m, prm);
        for (int j = 0; j <= K; j++)
            for (int i = 1; i <= W; i++)
                h[t * per_axis + size_t(j) * W + (i - 1)] =
                    psi_host(p->window, double(j) / K + double(m - i), m, prm) / psi0;
    }
    const size_t bytes = h.size() * p->rsize;
    std::vector<float> hf;
    const void *src = h.data();
    if (p->dtype == NFFT_FP32) {
        hf.assign(h.begin(), h.end());
        src = hf.data();
    }
    cudaError_t e = dev_alloc(&p->lin_tab, bytes, "lin");
    if (e == cudaSuccess) e = cudaMemcpy(p->lin_tab, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (p->lin_tab) cudaFree(p->lin_tab);
        p->lin_tab = nullptr;
        return e == cudaErrorMemoryAllocation ? NFFT_ENOMEM : NFFT_ECUDA;
    }
    g.lin = p->lin_tab;
    g.lin_k = K;
    return NFFT_OK;
}

// Host image of the tables below off_status (the layout is fixed by d, N, n, m and precision).
static void fill_tables(const gbnfft_plan *p, char *host)
{
    const bool fp64 = p->dtype == NFFT_FP64;
    const int m = p->m;
    const int deg = poly_degree(fp64, m);
    const size_t poly_axis = size_t(poly_axis_stride(fp64, m));
    for (int t = 0; t < p->d; t++) {
        const double prm = p->geom.win[t].prm;
        const double psi0 = psi_host(p->window, 0.0, m, prm);
        // psi_t(0) / (n_t phihat_t(k)): the per-axis factor of 1 / (|I_n| c_k) (Algorithm
        // "NFFT", deconvolution step) for the window normalised to psibar(0) = 1
        for (int64_t i = 0; i < p->N[t]; i++) {
            const double k = double(i - p->N[t] / 2);
            const double dc = psi0 / nphihat_host(p->window, k, double(p->n[t]), m, prm);
            if (fp64)
                reinterpret_cast<double *>(host + p->off_dc[t])[i] = dc;
            else
                reinterpret_cast<float *>(host + p->off_dc[t])[i] = (float)dc;
        }
        // window polynomials of this axis: coefficient k of tap i at [k * kPolyTaps + i - 1]
        for (int i = 1; i <= 2 * m; i++) {
            double mono[32];
            fit_tap_poly(p->window, m, prm, i, deg, mono);
            for (int k = 0; k <= deg; k++) {
                const size_t e = size_t(t) * poly_axis + size_t(k) * kPolyTaps + size_t(i - 1);
                if (fp64)
                    reinterpret_cast<double *>(host + p->off_poly)[e] = mono[k];
                else
                    reinterpret_cast<float *>(host + p->off_poly)[e] = (float)mono[k];
            }
        }
        for (int64_t j = 0; j < p->n[t]; j++) {
            double re, im;
            twiddle(j, p->n[t], &re, &im);
            if (fp64)
                reinterpret_cast<double2 *>(host + p->off_tw[t])[j] = make_double2(re, im);
            else
                reinterpret_cast<float2 *>(host + p->off_tw[t])[j] =
                    make_float2((float)re, (float)im);
        }
        if (p->blu_M[t]) {
            // chirp w_j = e^(-pi i j^2 / L) = e^(-2 pi i (j^2 mod 2L) / (2L)), exact reduction
            const int64_t L = p->n[t], Mb = p->blu_M[t];
            std::vector<std::complex<double>> w(L), vf(Mb, 0.0), vi(Mb, 0.0);
            for (int64_t j = 0; j < L; j++) {
                double re, im;
                twiddle((j * j) % (2 * L), 2 * L, &re, &im);
                w[j] = std::complex<double>(re, im);
            }
            // wrapped filters: v_m for |m| < L at index m mod M; forward uses conj(w)
            for (int64_t j = 0; j < L; j++) {
                vf[j] = std::conj(w[j]);
                vi[j] = w[j];
                if (j > 0) {
                    vf[Mb - j] = std::conj(w[j]);
                    vi[Mb - j] = w[j];
                }
            }
            host_fft_pow2(vf);
            host_fft_pow2(vi);
            for (int64_t j = 0; j < Mb; j++) {
                double re, im;
                twiddle(j, Mb, &re, &im);
                const std::complex<double> a = vf[j] / double(Mb), b = vi[j] / double(Mb);
                if (fp64) {
                    put_complex<double2, double>(host + p->off_ff[t], j, a.real(), a.imag());
                    put_complex<double2, double>(host + p->off_fi[t], j, b.real(), b.imag());
                    put_complex<double2, double>(host + p->off_twM[t], j, re, im);
                } else {
                    put_complex<float2, float>(host + p->off_ff[t], j, a.real(), a.imag());
                    put_complex<float2, float>(host + p->off_fi[t], j, b.real(), b.imag());
                    put_complex<float2, float>(host + p->off_twM[t], j, re, im);
                }
            }
            for (int64_t j = 0; j < L; j++) {
                if (fp64)
                    put_complex<double2, double>(host + p->off_chirp[t], j, w[j].real(),
                                                 w[j].imag());
                else
                    put_complex<float2, float>(host + p->off_chirp[t], j, w[j].real(),
                                               w[j].imag());
            }
        }
    }
}

// Host copy of the window polynomials (the kernels that take them as an argument copy it at
// every launch).
static void keep_poly_host(gbnfft_plan *p, const char *host)
{
    const size_t bytes = size_t(p->d) * poly_axis_stride(p->dtype == NFFT_FP64, p->m) * p->rsize;
    p->poly_host.assign(host + p->off_poly, host + p->off_poly + bytes);
    p->geom.poly_host = p->poly_host.data();
}

// Switch the window: new edge constants and tables, written over the old ones in place (the
// device pointers, the status word and the node preprocessing stay valid).
static int set_window(gbnfft_plan *p, int kind)
{
    if (kind == p->window) return NFFT_OK;
    const int old = p->window;
    p->window = kind;
    set_window_constants(p);
    char *host = static_cast<char *>(std::calloc(1, p->tbytes));
    if (!host) {
        p->window = old;
        set_window_constants(p);
        return NFFT_ENOMEM;
    }
    fill_tables(p, host);
    keep_poly_host(p, host);
    // the old tables may be read by work queued on any stream of the device
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(p->tables, host, p->off_status, cudaMemcpyHostToDevice);
    std::free(host);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return NFFT_ECUDA;
    }
    return build_lin_tables(p);  // the lookup tables follow the window (no-op when off)
}

int nfft_plan_create(nfft_plan *out, int d, const int64_t *N, int64_t M, const int64_t *n, int m,
                     int dtype)
{
    if (!out) return NFFT_EINVAL;
    *out = nullptr;
    if (d < 1 || d > 3 || !N) return NFFT_EINVAL;
    if (dtype != NFFT_FP32 && dtype != NFFT_FP64) return NFFT_EINVAL;
    if (M < 0 || M > 0x7fffffffLL) return NFFT_EINVAL;
    if (m <= 0) m = 8;
    int64_t nn[3] = {0, 0, 0}, NNv[3] = {0, 0, 0};
    for (int t = 0; t < d; t++) {
        NNv[t] = N[t];
        if (N[t] < 2 || (N[t] & 1)) return NFFT_EINVAL;
        if (N[t] > (int64_t(1) << 30)) return NFFT_EUNSUPPORTED;
        nn[t] = n ? n[t] : (int64_t(1) << (ilog2(N[t]) + 1));
        if (nn[t] <= N[t] || (nn[t] & 1)) return NFFT_EINVAL;
        if (2 * int64_t(m) + 2 > nn[t]) return NFFT_EINVAL;
    }
    if (m > kMaxM) return NFFT_EUNSUPPORTED;
    int64_t G = 1, NN = 1;
    int cbits = 0;
    for (int t = 0; t < d; t++) {
        // powers of two up to 16384 (FP32) / 8192 (FP64); other even lengths (Bluestein, whose
        // power-of-two convolution length is at most 8192 / 4096) up to 4096 / 2048
        if (is_pow2(nn[t])) {
            if (nn[t] > (dtype == NFFT_FP32 ? 16384 : 8192)) return NFFT_EUNSUPPORTED;
        } else {
            if (nn[t] > (dtype == NFFT_FP32 ? 4096 : 2048)) return NFFT_EUNSUPPORTED;
        }
        G *= nn[t];
        NN *= NNv[t];
        cbits += ilog2(nn[t]);
    }
    if (G > 0x7fffffffLL || cbits > 31) return NFFT_EUNSUPPORTED;

    gbnfft_plan *p = new (std::nothrow) gbnfft_plan();
    if (!p) return NFFT_ENOMEM;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return NFFT_ECUDA;
    }
    p->d = d;
    p->m = m;
    p->dtype = dtype;
    p->M = M;
    p->G = G;
    p->NN = NN;
    p->csize = dtype == NFFT_FP32 ? sizeof(float2) : sizeof(double2);
    p->rsize = dtype == NFFT_FP32 ? sizeof(float) : sizeof(double);
    for (int t = 0; t < d; t++) {
        p->N[t] = NNv[t];
        p->n[t] = nn[t];
    }
    // second FFT buffer: the largest intermediate that cannot live in gA
    if (d == 2) p->Bsz = NNv[0] * nn[1];
    if (d == 3) p->Bsz = NNv[0] * nn[1] * nn[2];

    // geometry, window constants and bins
    Geom &g = p->geom;
    g.d = d;
    g.m = m;
    g.spread_method = kSpreadAuto;
    g.interp_method = kInterpAuto;
    for (int t = 0; t < kMaxDim; t++) {
        if (t >= d) {
            g.n[t] = 1;
            g.cbits[t] = 0;
            g.cmask[t] = 0;
            g.N[t] = 1;
            g.win[t] = AxisWin{0.0, 0.0, 0.0};
            continue;
        }
        g.n[t] = (int)nn[t];
        g.cbits[t] = ilog2(nn[t]);
        g.cmask[t] = (1 << g.cbits[t]) - 1;
        if (!is_pow2(nn[t])) {  // Bluestein: convolution length and scratch (lines x M)
            p->blu_M[t] = 1 << ilog2(2 * nn[t] - 1);
            p->blu_elems = std::max(p->blu_elems, size_t(G / nn[t]) * size_t(p->blu_M[t]));
        }
        g.N[t] = (int)NNv[t];
    }
    set_window_constants(p);
    setup_bins(p);

    // tables: deconvolution factors and twiddles per axis, window polynomials, status word
    size_t tbytes = 0;
    for (int t = 0; t < d; t++) {
        p->off_dc[t] = tbytes;
        tbytes = align_up(tbytes + size_t(NNv[t]) * p->rsize, 256);
        p->off_tw[t] = tbytes;
        tbytes = align_up(tbytes + size_t(nn[t]) * p->csize, 256);
        if (p->blu_M[t]) {
            const int Mb = p->blu_M[t];
            p->off_chirp[t] = tbytes;
            tbytes = align_up(tbytes + size_t(nn[t]) * p->csize, 256);
            p->off_ff[t] = tbytes;
            tbytes = align_up(tbytes + size_t(Mb) * p->csize, 256);
            p->off_fi[t] = tbytes;
            tbytes = align_up(tbytes + size_t(Mb) * p->csize, 256);
            p->off_twM[t] = tbytes;
            tbytes = align_up(tbytes + size_t(Mb) * p->csize, 256);
        }
    }
    p->off_poly = tbytes;
    tbytes = align_up(tbytes + size_t(d) * poly_axis_stride(dtype == NFFT_FP64, m) * p->rsize, 256);
    p->off_status = tbytes;
    tbytes += 256;
    p->tbytes = tbytes;
    char *host = static_cast<char *>(std::calloc(1, tbytes));
    if (!host) {
        delete p;
        return NFFT_ENOMEM;
    }
    fill_tables(p, host);
    keep_poly_host(p, host);
    cudaError_t e = dev_alloc(&p->tables, tbytes, "tables");
    if (e == cudaSuccess) e = cudaMemcpy(p->tables, host, tbytes, cudaMemcpyHostToDevice);
    std::free(host);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (p->tables) cudaFree(p->tables);
        delete p;
        return e == cudaErrorMemoryAllocation ? NFFT_ENOMEM : NFFT_ECUDA;
    }
    char *tb = static_cast<char *>(p->tables);
    for (int t = 0; t < d; t++) {
        p->deconv[t] = tb + p->off_dc[t];
        p->tw[t] = tb + p->off_tw[t];
    }
    p->d_status = reinterpret_cast<int *>(tb + p->off_status);
    g.poly = tb + p->off_poly;
    *out = p;
    return NFFT_OK;
}

int nfft_destroy(nfft_plan p)
{
    if (!p) return NFFT_OK;
    set_device(p);
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    if (p->tables) cudaFree(p->tables);
    if (p->lin_tab) cudaFree(p->lin_tab);
    if (p->ws_owned && p->ws) cudaFree(p->ws);
    if (p->stage) cudaFree(p->stage);
    for (auto &pp : p->prof) {
        cudaEventDestroy(pp.a);
        cudaEventDestroy(pp.b);
    }
    delete p;
    return NFFT_OK;
}

int nfft_set_stream(nfft_plan p, void *stream)
{
    if (!p) return NFFT_EINVAL;
    p->stream = static_cast<cudaStream_t>(stream);
    return NFFT_OK;
}

int nfft_workspace_size(nfft_plan p, size_t *bytes)
{
    if (!p || !bytes) return NFFT_EINVAL;
    *bytes = p->ws_need;
    return NFFT_OK;
}

int nfft_set_workspace(nfft_plan p, void *ptr, size_t bytes)
{
    if (!p || !ptr) return NFFT_EINVAL;
    if (!aligned(ptr, 256)) return NFFT_EINVAL;
    if (bytes < p->ws_need) return NFFT_ENOMEM;
    if (p->ws_owned && p->ws) {
        set_device(p);
        if (p->stream) cudaStreamSynchronize(p->stream);
        cudaFree(p->ws);
    }
    p->ws = static_cast<char *>(ptr);
    p->ws_bytes = bytes;
    p->ws_owned = false;
    p->nodes_ready = false;  // the sorted node data lived in the old workspace
    return NFFT_OK;
}

int nfft_get_info(nfft_plan p, nfft_info *info)
{
    if (!p || !info) return NFFT_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->d = p->d;
    info->m = p->m;
    info->dtype = p->dtype;
    info->M = p->M;
    for (int t = 0; t < p->d; t++) {
        info->N[t] = p->N[t];
        info->n[t] = p->n[t];
        info->bin[t] = p->geom.bs[t];
    }
    info->workspace_bytes = p->ws_need;
    info->window = p->window;
    info->window_table = p->lin_k;
    return NFFT_OK;
}

int nfft_set_nodes(nfft_plan p, const void *x)
{
    if (!p) return NFFT_EINVAL;
    if (p->M > 0 && (!x || !aligned(x, p->rsize))) return NFFT_EINVAL;
    int rc = set_device(p);
    if (rc) return rc;
    rc = ensure_workspace(p);
    if (rc) return rc;
    if (p->ws_bytes < p->ws_need) return NFFT_ENOMEM;
    p->nodes_ready = false;
    rc = p->dtype == NFFT_FP32 ? do_set_nodes<float>(p, x) : do_set_nodes<double>(p, x);
    if (rc) return rc;
    p->nodes_ready = true;
    return NFFT_OK;
}

int nfft_trafo(nfft_plan p, const void *fhat, void *f)
{
    if (!p) return NFFT_EINVAL;
    if (!p->nodes_ready) return NFFT_ENOTREADY;
    if (check_dev_ptr(p, fhat, p->NN) || check_dev_ptr(p, f, p->M)) return NFFT_EINVAL;
    int rc = set_device(p);
    if (rc) return rc;
    if (p->M == 0) return NFFT_OK;
    return p->dtype == NFFT_FP32 ? do_trafo<float>(p, fhat, f) : do_trafo<double>(p, fhat, f);
}

int nfft_adjoint(nfft_plan p, const void *f, void *fhat)
{
    if (!p) return NFFT_EINVAL;
    if (!p->nodes_ready) return NFFT_ENOTREADY;
    if (check_dev_ptr(p, f, p->M) || check_dev_ptr(p, fhat, p->NN)) return NFFT_EINVAL;
    int rc = set_device(p);
    if (rc) return rc;
    if (p->M == 0) {
        GB_CHECK(cudaMemsetAsync(fhat, 0, size_t(p->NN) * p->csize, p->stream));
        return NFFT_OK;
    }
    return p->dtype == NFFT_FP32 ? do_adjoint<float>(p, f, fhat) : do_adjoint<double>(p, f, fhat);
}

int nfft_grad_x(nfft_plan p, const void *coef, const void *w, void *gx)
{
    if (!p) return NFFT_EINVAL;
    if (!p->nodes_ready) return NFFT_ENOTREADY;
    if (check_dev_ptr(p, coef, p->NN) || check_dev_ptr(p, w, p->M)) return NFFT_EINVAL;
    if (p->M > 0 && (!gx || !aligned(gx, p->rsize))) return NFFT_EINVAL;
    int rc = set_device(p);
    if (rc) return rc;
    if (p->M == 0) return NFFT_OK;
    return p->dtype == NFFT_FP32 ? do_grad<float>(p, coef, w, gx) : do_grad<double>(p, coef, w, gx);
}

int nfft_status(nfft_plan p)
{
    if (!p) return NFFT_EINVAL;
    int rc = set_device(p);
    if (rc) return rc;
    cudaError_t e = p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return NFFT_ECUDA;
    int h = 0;
    if (cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return NFFT_ECUDA;
    if (h != 0) {
        const int zero = 0;
        if (cudaMemcpy(p->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            return NFFT_ECUDA;
    }
    return h;
}

int nfft_set_option(nfft_plan p, int key, int64_t value)
{
    if (!p) return NFFT_EINVAL;
    switch (key) {
    case NFFT_OPT_SPREAD_METHOD:
        if (value < kSpreadAuto || value > kSpreadRows) return NFFT_EINVAL;
        p->geom.spread_method = (int)value;
        return NFFT_OK;
    case NFFT_OPT_INTERP_METHOD:
        if (value < kInterpAuto || value > kInterpOctet) return NFFT_EINVAL;
        p->geom.interp_method = (int)value;
        return NFFT_OK;
    case NFFT_OPT_WINDOW:
        if (value < kWinKB || value > kWinSinc) return NFFT_EINVAL;
        set_device(p);
        return set_window(p, (int)value);
    case NFFT_OPT_WINDOW_TABLE: {
        if (value < 0 || value == 1 || value > 65536) return NFFT_EINVAL;
        set_device(p);
        const int old = p->lin_k;
        p->lin_k = (int)value;
        set_window_constants(p);
        const int rc = build_lin_tables(p);
        if (rc) {
            p->lin_k = old;
            set_window_constants(p);
            build_lin_tables(p);
        }
        return rc;
    }
    case NFFT_OPT_STRIPE_ITEM: {
        if (value < 0 || value > 65536 || (value > 0 && (value < 8 || !is_pow2(value))))
            return NFFT_EINVAL;
        p->stripe_item_req = value;
        const size_t old_need = p->ws_need;
        setup_bins(p);
        p->nodes_ready = false;  // the item list is built by set_nodes
        if (p->ws_owned && p->ws && p->ws_need > old_need) {
            set_device(p);
            if (p->stream) cudaStreamSynchronize(p->stream);
            cudaFree(p->ws);
            p->ws = nullptr;
            p->ws_bytes = 0;
            p->ws_owned = false;
        }
        return NFFT_OK;
    }
    case NFFT_OPT_SUBPROBLEM: {
        if (value < 0 || value > kMaxSub || (value > 0 && (value < 32 || !is_pow2(value))))
            return NFFT_EINVAL;
        p->sub_req = value;
        const size_t old_need = p->ws_need;
        setup_bins(p);
        p->nodes_ready = false;  // the subproblem list is built by set_nodes
        if (p->ws_owned && p->ws && p->ws_need > old_need) {
            set_device(p);
            if (p->stream) cudaStreamSynchronize(p->stream);
            cudaFree(p->ws);
            p->ws = nullptr;
            p->ws_bytes = 0;
            p->ws_owned = false;
        }
        return NFFT_OK;
    }
    case NFFT_OPT_BIN_0:
    case NFFT_OPT_BIN_1:
    case NFFT_OPT_BIN_2: {
        const int t = key - NFFT_OPT_BIN_0;
        if (t >= p->d) return NFFT_EINVAL;
        if (value < 0 || (value > 0 && !is_pow2(value))) return NFFT_EINVAL;
        {
            // the spreading tile (bin + 2m halo per axis, complex) must fit in shared memory
            size_t cells = 1;
            for (int u = 0; u < p->d; u++) {
                int64_t bs = u == t ? value : p->geom.bs[u];
                if (u == t && value == 0) bs = 0;  // default: always fits
                if (bs == 0) {
                    cells = 0;
                    break;
                }
                if (bs > p->n[u]) bs = p->n[u];
                cells *= size_t(bs + 2 * p->m);
            }
            // 227 KB per CTA minus the window tables kept beside the tile
            const size_t tables = size_t(kMaxDim) * poly_axis_stride(p->dtype == NFFT_FP64, p->m) *
                                  p->rsize;
            if (cells * p->csize > 227 * 1024 - tables) return NFFT_EINVAL;
        }
        p->bin_req[t] = value;
        const size_t old_need = p->ws_need;
        setup_bins(p);
        p->nodes_ready = false;  // the node order depends on the bins
        if (p->ws_owned && p->ws && p->ws_need > old_need) {
            set_device(p);
            if (p->stream) cudaStreamSynchronize(p->stream);
            cudaFree(p->ws);
            p->ws = nullptr;
            p->ws_bytes = 0;
            p->ws_owned = false;
        }
        return NFFT_OK;
    }
    default:
        return NFFT_EINVAL;
    }
}

int nfft_profile(nfft_plan p, int enable)
{
    if (!p) return NFFT_EINVAL;
    p->prof_on = enable != 0;
    p->prof_used = 0;
    return NFFT_OK;
}

int nfft_profile_read(nfft_plan p, double *ms, int64_t *count, int nstages)
{
    if (!p || !ms || nstages < 0) return NFFT_EINVAL;
    int rc = set_device(p);
    if (rc) return rc;
    for (int i = 0; i < nstages; i++) {
        ms[i] = 0.0;
        if (count) count[i] = 0;
    }
    GB_CHECK(p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize());
    for (size_t i = 0; i < p->prof_used; i++) {
        const auto &pp = p->prof[i];
        if (pp.stage < 0 || pp.stage >= nstages) continue;
        float t = 0.f;
        GB_CHECK(cudaEventElapsedTime(&t, pp.a, pp.b));
        ms[pp.stage] += t;
        if (count) count[pp.stage] += 1;
    }
    p->prof_used = 0;
    return NFFT_OK;
}

// ---------------------------------------------------------------------------- host variants

static int ensure_stage(gbnfft_plan *p)
{
    // x (M d reals), fhat (|I_N| complex), f (M complex), each 256-byte aligned
    const size_t bx = align_up(size_t(p->M) * p->d * p->rsize, 256);
    const size_t bh = align_up(size_t(p->NN) * p->csize, 256);
    const size_t bf = align_up(size_t(p->M) * p->csize, 256);
    const size_t need = bx + bh + bf;
    if (p->stage && p->stage_bytes >= need) return NFFT_OK;
    if (p->stage) cudaFree(p->stage);
    p->stage = nullptr;
    if (dev_alloc(&p->stage, need, "stage") != cudaSuccess) {
        cudaGetLastError();
        p->stage_bytes = 0;
        return NFFT_ENOMEM;
    }
    p->stage_bytes = need;
    return NFFT_OK;
}

static char *stage_x(gbnfft_plan *p) { return static_cast<char *>(p->stage); }
static char *stage_fhat(gbnfft_plan *p)
{
    return stage_x(p) + align_up(size_t(p->M) * p->d * p->rsize, 256);
}
static char *stage_f(gbnfft_plan *p)
{
    return stage_fhat(p) + align_up(size_t(p->NN) * p->csize, 256);
}

int nfft_set_nodes_host(nfft_plan p, const void *x_host)
{
    if (!p) return NFFT_EINVAL;
    if (p->M > 0 && !x_host) return NFFT_EINVAL;
    int rc = set_device(p);
    if (rc) return rc;
    rc = ensure_stage(p);
    if (rc) return rc;
    const size_t bytes = size_t(p->M) * p->d * p->rsize;
    if (bytes) GB_CHECK(cudaMemcpyAsync(stage_x(p), x_host, bytes, cudaMemcpyHostToDevice,
                                        p->stream));
    rc = nfft_set_nodes(p, stage_x(p));
    if (rc) return rc;
    GB_CHECK(p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize());
    return NFFT_OK;
}

int nfft_trafo_host(nfft_plan p, const void *fhat_host, void *f_host)
{
    if (!p) return NFFT_EINVAL;
    if (!p->nodes_ready) return NFFT_ENOTREADY;
    if ((p->NN > 0 && !fhat_host) || (p->M > 0 && !f_host)) return NFFT_EINVAL;
    int rc = set_device(p);
    if (rc) return rc;
    rc = ensure_stage(p);
    if (rc) return rc;
    GB_CHECK(cudaMemcpyAsync(stage_fhat(p), fhat_host, size_t(p->NN) * p->csize,
                             cudaMemcpyHostToDevice, p->stream));
    rc = nfft_trafo(p, stage_fhat(p), stage_f(p));
    if (rc) return rc;
    if (p->M) GB_CHECK(cudaMemcpyAsync(f_host, stage_f(p), size_t(p->M) * p->csize,
                                       cudaMemcpyDeviceToHost, p->stream));
    GB_CHECK(p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize());
    return NFFT_OK;
}

int nfft_adjoint_host(nfft_plan p, const void *f_host, void *fhat_host)
{
    if (!p) return NFFT_EINVAL;
    if (!p->nodes_ready) return NFFT_ENOTREADY;
    if ((p->NN > 0 && !fhat_host) || (p->M > 0 && !f_host)) return NFFT_EINVAL;
    int rc = set_device(p);
    if (rc) return rc;
    rc = ensure_stage(p);
    if (rc) return rc;
    if (p->M) GB_CHECK(cudaMemcpyAsync(stage_f(p), f_host, size_t(p->M) * p->csize,
                                       cudaMemcpyHostToDevice, p->stream));
    rc = nfft_adjoint(p, stage_f(p), stage_fhat(p));
    if (rc) return rc;
    GB_CHECK(cudaMemcpyAsync(fhat_host, stage_fhat(p), size_t(p->NN) * p->csize,
                             cudaMemcpyDeviceToHost, p->stream));
    GB_CHECK(p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize());
    return NFFT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------ batches
// A batch runs many independent plans (uneven N and M) concurrently: every call forks the
// batch's stream into a few side streams with one event, issues plan i on side stream lane[i]
// (the plan's own stream is swapped for the duration of the call), and joins the side streams
// back with one event each. Plans go to lanes largest first, each to the lane with the least
// work so far (work ~ M + |I_n|). The pattern records into a CUDA graph as parallel branches.
//
// A batch whose plans qualify is run fused instead (see batch_fused.cu): one launch per stage
// over all plans, in the batch's stream, from per-plan tables and work lists kept in one device
// block (uploaded from pinned host memory, waited for once). The tables are rebuilt when a
// plan's workspace or tuning changed since they were built.
enum FusedPass { kFwdRows = 0, kFwdCols = 1, kAdjCols = 2, kAdjRows = 3, kFusedPasses = 4 };

struct FusedSig {  // the plan state the fused tables depend on
    const void *ws;
    int bs[3], spread, interp, lin_k, window;
    bool operator==(const FusedSig &o) const
    {
        return ws == o.ws && bs[0] == o.bs[0] && bs[1] == o.bs[1] && bs[2] == o.bs[2] &&
               spread == o.spread && interp == o.interp && lin_k == o.lin_k &&
               window == o.window;
    }
};

struct gbnfft_batch {
    std::vector<gbnfft_plan *> plans;
    std::vector<int> lane;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    // fused execution
    bool fused = false;           // run fused (requested and the plans qualify)
    bool fused_wanted = true;
    std::vector<FusedSig> sig;    // per plan, when the tables were built
    char *fdev = nullptr;         // device block: node plans, passes, items, prefix, counters
    char *fhost = nullptr;        // pinned host image of the same block
    size_t fbytes = 0;
    size_t off_nodes = 0, off_pass[kFusedPasses] = {}, off_items[kFusedPasses] = {};
    size_t off_istart = 0, off_work = 0;
    int nitems[kFusedPasses] = {};
    size_t fft_smem[kFusedPasses] = {};
    int node_blocks = 0, zero_blocks = 0, max_items = 0, tile_cells = 0;
    bool shared_window = false;  // every plan has the same window polynomials
    int rows_bs0 = 0, rows_g = 0;  // rows-form spreading (bin rows, lanes per tile), 0: half-warp
    FusedOffsets offsets{};      // per-plan first blocks of the per-node and zeroing stages
};

namespace {

void batch_free(gbnfft_batch *b)
{
    for (cudaStream_t s : b->side)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->fdev) cudaFree(b->fdev);
    if (b->fhost) cudaFreeHost(b->fhost);
    delete b;
}

FusedSig fused_sig(const gbnfft_plan *p)
{
    FusedSig s{};
    s.ws = p->ws;
    for (int t = 0; t < 3; t++) s.bs[t] = p->geom.bs[t];
    s.spread = p->geom.spread_method;
    s.interp = p->geom.interp_method;
    s.lin_k = p->lin_k;
    s.window = p->window;
    return s;
}

// Whether the plans can run fused: 2-D FP32, one m and window, the half-warp or automatic
// spreading form and the thread interpolation form (automatic or chosen), polynomial window,
// power-of-two FFT lengths 16..4096.
bool fusable(const gbnfft_batch *b)
{
    const auto &ps = b->plans;
    if (ps.empty() || ps.size() > size_t(kFusedMax)) return false;
    const gbnfft_plan *p0 = ps[0];
    size_t cells = 0;
    for (const gbnfft_plan *p : ps) {
        if (p->d != 2 || p->dtype != NFFT_FP32 || p->m != p0->m || p->window != p0->window ||
            p->lin_k != 0)
            return false;
        if (p->geom.spread_method != kSpreadAuto && p->geom.spread_method != kSpreadHalf)
            return false;
        if (p->geom.interp_method != kInterpAuto && p->geom.interp_method != kInterpThread)
            return false;
        for (int t = 0; t < 2; t++)
            if (!is_pow2(p->n[t]) || p->n[t] < 16 || p->n[t] > 4096 || p->blu_M[t]) return false;
        cells = std::max(cells, size_t(half_tile_cells_f32(p->m, p->geom.bs[0], p->geom.bs[1])));
    }
    // private tiles and staging of the half-warp form in shared memory, beside static data
    return half_smem_bytes_f32(p0->m, (int)cells) <= 200 * 1024;
}

// Row stride (cells) of a line buffer of the radix-8 FFT for P lines of L (as launch_fftr).
int fused_ls(int L, int P, bool strided)
{
    int LS = 2 * (L + L / 16);
    if (strided && P > 1) {
        const int cells = 128 / (int)sizeof(float2);
        const int want = (cells / P) % cells;
        LS += ((want - LS % cells) + cells) % cells;
    }
    return LS;
}

// (Re)build the fused tables from the plans' current state and enqueue their upload.
int fused_build(gbnfft_batch *b)
{
    const int n = (int)b->plans.size();
    std::vector<FusedNodePlan> nodes(n);
    std::vector<FusedFftPass> pass[kFusedPasses];
    std::vector<FusedItem> items[kFusedPasses];
    int node_blocks = 0, zero_blocks = 0, max_items = 0, cells = 0;
    for (int i = 0; i < n; i++) {
        gbnfft_plan *p = b->plans[i];
        FusedNodePlan &q = nodes[i];
        std::memset(&q, 0, sizeof(q));
        q.g = p->geom;
        q.g.sw = StripeWork{};
        q.grid = at<float2>(p, p->gA);
        q.fgrid = at<float2>(p, p->gC);
        q.rec = at<RecF>(p, p->rec);
        q.perm = at<int>(p, p->perm);
        q.subs = at<SubProb>(p, p->subs);
        q.nsub = at<int>(p, p->nsub);
        q.M = (int)p->M;
        q.G = p->G;
        b->offsets.node_block0[i] = node_blocks;
        b->offsets.zero_block0[i] = zero_blocks;
        node_blocks += (int)((p->M + 127) / 128);
        zero_blocks += zero_fused_blocks(p->G, sizeof(float2));
        max_items += p->max_subs;
        cells = std::max(cells, half_tile_cells_f32(p->m, p->geom.bs[0], p->geom.bs[1]));
        // the four pruned passes of Algorithm "NFFT" (rows then columns, D fused) and of
        // Algorithm "adjoint NFFT" (columns then rows, D^H fused)
        float2 *A = at<float2>(p, p->gA), *B = at<float2>(p, p->gB);
        float2 *Cf = at<float2>(p, p->gC), *Df = at<float2>(p, p->gD);  // forward buffers
        const int n0 = (int)p->n[0], n1 = (int)p->n[1], N0 = (int)p->N[0], N1 = (int)p->N[1];
        const int Pr = kFusedFftThreads * 8 / n1, Pc = kFusedFftThreads * 8 / n0;
        const FusedFftPass q4[kFusedPasses] = {
            {nullptr, Df, N0, 1, ilog2(n1), N1, Pr, fused_ls(n1, Pr, false), 1, p->tw[1],
             p->deconv[1]},
            {Df, Cf, 1, n1, ilog2(n0), N0, Pc, fused_ls(n0, Pc, true), 1, p->tw[0],
             p->deconv[0]},
            {A, B, 1, n1, ilog2(n0), N0, Pc, fused_ls(n0, Pc, true), 0, p->tw[0], p->deconv[0]},
            {B, nullptr, N0, 1, ilog2(n1), N1, Pr, fused_ls(n1, Pr, false), 0, p->tw[1],
             p->deconv[1]}};
        for (int k = 0; k < kFusedPasses; k++) {
            const FusedFftPass &f = q4[k];
            pass[k].push_back(f);
            const long long blocks = f.inner == 1 ? (f.outer + f.P - 1) / f.P
                                                  : f.outer * ((f.inner + f.P - 1) / f.P);
            for (long long blk = 0; blk < blocks; blk++) items[k].push_back({i, (int)blk});
            b->fft_smem[k] = std::max(b->fft_smem[k], size_t(f.P) * f.LS * sizeof(float2));
        }
    }
    // one block: node plans, passes and items of the four passes, item prefix, counters
    size_t off = 0;
    auto put = [&](size_t bytes) {
        off = align_up(off, 256);
        const size_t at0 = off;
        off += bytes;
        return at0;
    };
    b->off_nodes = put(n * sizeof(FusedNodePlan));
    for (int k = 0; k < kFusedPasses; k++) {
        b->off_pass[k] = put(n * sizeof(FusedFftPass));
        b->off_items[k] = put(items[k].size() * sizeof(FusedItem));
        b->nitems[k] = (int)items[k].size();
    }
    b->off_istart = put((n + 1) * sizeof(int));
    b->off_work = put(4 * sizeof(int));
    const size_t need = align_up(off, 256);
    if (need > b->fbytes) {
        if (b->fdev) {
            cudaStreamSynchronize(b->stream);
            cudaFree(b->fdev);
            cudaFreeHost(b->fhost);
            b->fdev = nullptr;
            b->fhost = nullptr;
            b->fbytes = 0;
        }
        void *d = nullptr, *h = nullptr;
        if (dev_alloc(&d, need, "batch") != cudaSuccess) {
            cudaGetLastError();
            return NFFT_ENOMEM;
        }
        if (cudaMallocHost(&h, need) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(d);
            return NFFT_ENOMEM;
        }
        b->fdev = static_cast<char *>(d);
        b->fhost = static_cast<char *>(h);
        b->fbytes = need;
    } else {
        // the pinned image may still be read by an upload in flight
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return NFFT_ECUDA;
    }
    std::memset(b->fhost, 0, need);
    std::memcpy(b->fhost + b->off_nodes, nodes.data(), n * sizeof(FusedNodePlan));
    for (int k = 0; k < kFusedPasses; k++) {
        std::memcpy(b->fhost + b->off_pass[k], pass[k].data(), n * sizeof(FusedFftPass));
        std::memcpy(b->fhost + b->off_items[k], items[k].data(),
                    items[k].size() * sizeof(FusedItem));
    }
    // complete before any stream uses the tables (later calls may come on another stream)
    GB_CHECK(cudaMemcpyAsync(b->fdev, b->fhost, need, cudaMemcpyHostToDevice, b->stream));
    GB_CHECK(cudaStreamSynchronize(b->stream));
    b->offsets.node_block0[n] = node_blocks;
    b->offsets.zero_block0[n] = zero_blocks;
    b->shared_window = true;
    for (int i = 1; i < n; i++)
        b->shared_window &= b->plans[i]->poly_host == b->plans[0]->poly_host;
    // the rows form when every plan spreads automatically with sort bins of one height (4 or 8
    // rows) and tiles at most 32 cells wide (16: a half-warp per tile)
    b->rows_bs0 = b->plans[0]->geom.bs[0];
    b->rows_g = 16;
    for (int i = 0; i < n; i++) {
        const gbnfft_plan *p = b->plans[i];
        const int td1 = p->geom.bs[1] + 2 * p->m;
        if (p->geom.spread_method != kSpreadAuto || p->geom.bs[0] != b->rows_bs0 || td1 > 32)
            b->rows_bs0 = 0;
        if (td1 > 16) b->rows_g = 32;
    }
    if (b->rows_bs0 != 4 && b->rows_bs0 != 8) b->rows_bs0 = 0;
    b->node_blocks = node_blocks;
    b->zero_blocks = zero_blocks;
    b->max_items = max_items;
    b->tile_cells = cells;
    b->sig.resize(n);
    for (int i = 0; i < n; i++) b->sig[i] = fused_sig(b->plans[i]);
    return NFFT_OK;
}

// Tables current for the plans' state (rebuilt if a plan changed); false if the plans no
// longer qualify (the call then runs plan by plan).
int fused_ready(gbnfft_batch *b, bool &use)
{
    use = false;
    if (!b->fused_wanted) return NFFT_OK;
    bool same = b->fdev && b->sig.size() == b->plans.size();
    for (size_t i = 0; same && i < b->plans.size(); i++)
        same = b->sig[i] == fused_sig(b->plans[i]);
    if (!same) {
        if (!fusable(b)) return NFFT_OK;
        const int rc = fused_build(b);
        if (rc) return rc;
    }
    use = true;
    return NFFT_OK;
}

template <typename P> P *fused_at(gbnfft_batch *b, size_t off)
{
    return reinterpret_cast<P *>(b->fdev + off);
}

int fused_fft(gbnfft_batch *b, int k, int sign, const FusedPtrs &ptrs)
{
    GB_CHECK(launch_fft_fused<float>(fused_at<FusedFftPass>(b, b->off_pass[k]),
                                     fused_at<FusedItem>(b, b->off_items[k]), b->nitems[k], sign,
                                     b->fft_smem[k], ptrs, b->stream));
    return NFFT_OK;
}

int fused_trafo(gbnfft_batch *b, const void *const *fhat, void *const *f)
{
    FusedPtrs ptrs{};
    for (size_t i = 0; i < b->plans.size(); i++) {
        ptrs.in[i] = fhat[i];
        ptrs.out[i] = f[i];
    }
    int rc = fused_fft(b, kFwdRows, -1, ptrs);
    if (!rc) rc = fused_fft(b, kFwdCols, -1, ptrs);
    if (rc) return rc;
    GB_CHECK(launch_interp_fused(fused_at<FusedNodePlan>(b, b->off_nodes), (int)b->plans.size(),
                                 b->offsets, b->plans[0]->geom, ptrs, false,
                                 b->shared_window, b->stream));
    return NFFT_OK;
}

int fused_adjoint(gbnfft_batch *b, const void *const *f, void *const *fhat)
{
    FusedPtrs ptrs{};
    for (size_t i = 0; i < b->plans.size(); i++) {
        ptrs.in[i] = f[i];
        ptrs.out[i] = fhat[i];
    }
    const int n = (int)b->plans.size();
    FusedNodePlan *nodes = fused_at<FusedNodePlan>(b, b->off_nodes);
    GB_CHECK(launch_zero_fused(nodes, n, b->offsets, sizeof(float2), b->stream));
    GB_CHECK(launch_spread_fused(nodes, n, fused_at<int>(b, b->off_istart),
                                 fused_at<int>(b, b->off_work), b->max_items, b->tile_cells,
                                 b->plans[0]->geom, ptrs, b->shared_window, b->rows_bs0,
                                 b->rows_g, b->stream));
    int rc = fused_fft(b, kAdjCols, +1, ptrs);
    if (!rc) rc = fused_fft(b, kAdjRows, +1, ptrs);
    return rc;
}

int fused_grad(gbnfft_batch *b, const void *const *coef, const void *const *w, void *const *gx)
{
    FusedPtrs ptrs{};
    for (size_t i = 0; i < b->plans.size(); i++) ptrs.in[i] = coef[i];
    int rc = fused_fft(b, kFwdRows, -1, ptrs);
    if (!rc) rc = fused_fft(b, kFwdCols, -1, ptrs);
    if (rc) return rc;
    for (size_t i = 0; i < b->plans.size(); i++) {
        ptrs.in[i] = w[i];
        ptrs.out[i] = gx[i];
    }
    GB_CHECK(launch_interp_fused(fused_at<FusedNodePlan>(b, b->off_nodes), (int)b->plans.size(),
                                 b->offsets, b->plans[0]->geom, ptrs, true,
                                 b->shared_window, b->stream));
    return NFFT_OK;
}

int batch_device(gbnfft_batch *b)
{
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return NFFT_ECUDA;
    if (cur != b->device && cudaSetDevice(b->device) != cudaSuccess) return NFFT_ECUDA;
    return NFFT_OK;
}

// fn(plan, i) for every plan of the batch on its lane; the batch stream waits for all of them.
// The side streams are always joined back (also after a failed call), and the first error is
// returned; plans after a failure are not issued.
template <typename Fn> int batch_run(gbnfft_batch *b, Fn fn)
{
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return NFFT_ECUDA;
    if (cur != b->device && cudaSetDevice(b->device) != cudaSuccess) return NFFT_ECUDA;
    if (cudaEventRecord(b->fork, b->stream) != cudaSuccess) return NFFT_ECUDA;
    int rc = NFFT_OK;
    for (cudaStream_t s : b->side)
        if (cudaStreamWaitEvent(s, b->fork, 0) != cudaSuccess) rc = NFFT_ECUDA;
    for (size_t i = 0; i < b->plans.size() && rc == NFFT_OK; i++) {
        gbnfft_plan *p = b->plans[i];
        cudaStream_t keep = p->stream;
        p->stream = b->side[b->lane[i]];
        rc = fn(p, i);
        p->stream = keep;
    }
    for (size_t j = 0; j < b->side.size(); j++) {
        if (cudaEventRecord(b->join[j], b->side[j]) != cudaSuccess ||
            cudaStreamWaitEvent(b->stream, b->join[j], 0) != cudaSuccess)
            rc = rc ? rc : NFFT_ECUDA;
    }
    return rc;
}

}  // namespace

extern "C" {

int nfft_batch_create(nfft_batch *out, const nfft_plan *plans, int count, int streams)
{
    if (!out || !plans || count < 1) return NFFT_EINVAL;
    *out = nullptr;
    for (int i = 0; i < count; i++) {
        if (!plans[i]) return NFFT_EINVAL;
        if (plans[i]->device != plans[0]->device) return NFFT_EINVAL;
    }
    // a plan listed twice would run on two side streams at once over one workspace
    {
        std::vector<const gbnfft_plan *> sorted(plans, plans + count);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return NFFT_EINVAL;
    }
    if (streams <= 0) streams = 8;
    if (streams > count) streams = count;
    if (streams > 64) streams = 64;
    gbnfft_batch *b = new (std::nothrow) gbnfft_batch;
    if (!b) return NFFT_ENOMEM;
    b->device = plans[0]->device;
    b->plans.assign(plans, plans + count);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess ||
        (cur != b->device && cudaSetDevice(b->device) != cudaSuccess)) {
        batch_free(b);
        return NFFT_ECUDA;
    }
    b->side.assign(streams, nullptr);
    b->join.assign(streams, nullptr);
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int j = 0; j < streams && ok; j++) {
        ok = cudaStreamCreateWithFlags(&b->side[j], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        batch_free(b);
        return NFFT_ECUDA;
    }
    std::vector<int> order(count);
    std::vector<double> work(count), load(streams, 0.0);
    for (int i = 0; i < count; i++) {
        order[i] = i;
        work[i] = double(plans[i]->M) + double(plans[i]->G);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work[a] > work[c]; });
    b->lane.assign(count, 0);
    for (int i : order) {
        int best = 0;
        for (int j = 1; j < streams; j++)
            if (load[j] < load[best]) best = j;
        b->lane[i] = best;
        load[best] += work[i];
    }
    *out = b;
    return NFFT_OK;
}

int nfft_batch_destroy(nfft_batch b)
{
    if (!b) return NFFT_EINVAL;
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != b->device) cudaSetDevice(b->device);
    for (cudaStream_t s : b->side)
        if (s) cudaStreamSynchronize(s);
    batch_free(b);
    return NFFT_OK;
}

int nfft_batch_set_stream(nfft_batch b, void *stream)
{
    if (!b) return NFFT_EINVAL;
    b->stream = static_cast<cudaStream_t>(stream);
    return NFFT_OK;
}

int nfft_batch_size(nfft_batch b, int *count, int *streams)
{
    if (!b) return NFFT_EINVAL;
    if (count) *count = (int)b->plans.size();
    if (streams) *streams = (int)b->side.size();
    return NFFT_OK;
}

int nfft_batch_lane(nfft_batch b, int i)
{
    if (!b || i < 0 || i >= (int)b->plans.size()) return -1;
    return b->lane[i];
}

int nfft_batch_trafo(nfft_batch b, const void *const *fhat, void *const *f)
{
    if (!b || !fhat || !f) return NFFT_EINVAL;
    for (size_t i = 0; i < b->plans.size(); i++) {
        const gbnfft_plan *p = b->plans[i];
        if (!p->nodes_ready) return NFFT_ENOTREADY;
        if (check_dev_ptr(p, fhat[i], p->NN) || check_dev_ptr(p, f[i], p->M)) return NFFT_EINVAL;
    }
    bool use = false;
    int rc = fused_ready(b, use);
    if (rc) return rc;
    if (use) {
        if (batch_device(b)) return NFFT_ECUDA;
        return fused_trafo(b, fhat, f);
    }
    return batch_run(b, [&](gbnfft_plan *p, size_t i) { return nfft_trafo(p, fhat[i], f[i]); });
}

int nfft_batch_adjoint(nfft_batch b, const void *const *f, void *const *fhat)
{
    if (!b || !f || !fhat) return NFFT_EINVAL;
    for (size_t i = 0; i < b->plans.size(); i++) {
        const gbnfft_plan *p = b->plans[i];
        if (!p->nodes_ready) return NFFT_ENOTREADY;
        if (check_dev_ptr(p, f[i], p->M) || check_dev_ptr(p, fhat[i], p->NN)) return NFFT_EINVAL;
    }
    bool use = false;
    int rc = fused_ready(b, use);
    if (rc) return rc;
    if (use) {
        if (batch_device(b)) return NFFT_ECUDA;
        return fused_adjoint(b, f, fhat);
    }
    return batch_run(b, [&](gbnfft_plan *p, size_t i) { return nfft_adjoint(p, f[i], fhat[i]); });
}

int nfft_batch_grad_x(nfft_batch b, const void *const *coef, const void *const *w,
                      void *const *gx)
{
    if (!b || !coef || !w || !gx) return NFFT_EINVAL;
    for (size_t i = 0; i < b->plans.size(); i++) {
        const gbnfft_plan *p = b->plans[i];
        if (!p->nodes_ready) return NFFT_ENOTREADY;
        if (check_dev_ptr(p, coef[i], p->NN) || check_dev_ptr(p, w[i], p->M)) return NFFT_EINVAL;
        if (p->M > 0 && (!gx[i] || !aligned(gx[i], p->rsize))) return NFFT_EINVAL;
    }
    bool use = false;
    int rc = fused_ready(b, use);
    if (rc) return rc;
    if (use) {
        if (batch_device(b)) return NFFT_ECUDA;
        return fused_grad(b, coef, w, gx);
    }
    return batch_run(b, [&](gbnfft_plan *p, size_t i) {
        return nfft_grad_x(p, coef[i], w[i], gx[i]);
    });
}

int nfft_batch_set_fused(nfft_batch b, int enable)
{
    if (!b) return NFFT_EINVAL;
    if (!enable) {
        b->fused_wanted = false;
        return NFFT_OK;
    }
    if (!fusable(b)) return NFFT_EUNSUPPORTED;
    b->fused_wanted = true;
    return NFFT_OK;
}

int nfft_batch_get_fused(nfft_batch b, int *fused)
{
    if (!b || !fused) return NFFT_EINVAL;
    *fused = (b->fused_wanted && fusable(b)) ? 1 : 0;
    return NFFT_OK;
}

}  // extern "C"
