/*
 * FP64 CPU oracle for the NFFT and the NDFT (Schmischke, "NFFT Interface for Julia",
 * arXiv 1810.09891, Sections 1 and 2).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the CUDA library is
 * checked against. Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it. It shares no code, header, table or constant with the CUDA library, and the
 * library never calls it.
 *
 * Conventions (Section 1, eq. NDFT; Section 2, eq. index_set):
 *   - complex arrays are interleaved (re, im) FP64, i.e. C99 double _Complex;
 *   - nodes x are stored (M, d) row-major, coordinate t pairs with frequency index k_t;
 *   - coefficients fhat are stored row-major over I_N, position k_t + N_t/2 on axis t
 *     (the centred order of the paper's Julia example, extended row-major to d > 1);
 *   - the oversampled grid g (|I_n| values) is stored row-major in natural FFT order:
 *     index l_t mod n_t on axis t.
 *
 * Readings of the paper used here (each is also listed with the design notes):
 *   - Kaiser-Bessel pair (the paper defers its formula to Plonka-Potts-Steidl-Tasche, Ch. 7.2):
 *       b = pi (2 - 1/sigma),  sigma = n/N,
 *       phi(x)    = sinh(b sqrt(m^2 - n^2 x^2)) / (pi sqrt(m^2 - n^2 x^2)),  |x| <= m/n,
 *       phihat(k) = (1/n) I0(m sqrt(b^2 - (2 pi k / n)^2)),                  |2 pi k/n| <= b.
 *     In grid units t = n x the window is psi(t) = phi(t/n).
 *   - The support of the truncated window (eq. window_cutoff, eq. Inm) is the closed interval
 *     |t| <= m. A node exactly on a grid point therefore has 2m+1 taps in that dimension,
 *     otherwise 2m.
 *   - The adjoint's spreading step (Algorithm "adjoint NFFT", first loop) sums over
 *     j in I^T_{n,m}(l); it is evaluated here by visiting every node once and adding its
 *     contributions (the same sum, in node order).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

static const double ORA_PI = 3.14159265358979323846264338327950288;

int ora_version(void) { return 1; }

int ora_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Number of OpenMP threads for later calls (n >= 1); returns the number in effect. */
int ora_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Small helpers                                                                              */
/* ------------------------------------------------------------------------------------------ */

static int64_t prod64(int d, const int64_t *v)
{
    int64_t p = 1;
    for (int t = 0; t < d; t++) p *= v[t];
    return p;
}

/* Non-negative remainder l mod n. */
static int64_t mod64(int64_t l, int64_t n)
{
    int64_t r = l % n;
    return r < 0 ? r + n : r;
}

/* Fractional part of k*x, reduced into about [-1/2, 1/2], with the rounding error of the
 * product recovered by an fma, so that e^{-2 pi i k x} is evaluated to full FP64 accuracy
 * even when |k x| is large. */
static double reduced_product(int64_t k, double x)
{
    double p = (double)k * x;
    double e = fma((double)k, x, -p);
    return (p - nearbyint(p)) + e;
}

/* ------------------------------------------------------------------------------------------ */
/* Direct transforms (Section 1, eq. NDFT and the adjoint sum after it)                        */
/* ------------------------------------------------------------------------------------------ */

/* f_j = sum_{k in I_N} fhat_k e^{-2 pi i k.x_j},  j = 0..M-1   (Section 1, eq. NDFT). */
void ora_ndft(int d, const int64_t *N, int64_t M, const double *x, const cplx *fhat, cplx *f)
{
    const int64_t nk = prod64(d, N);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < M; j++) {
        cplx acc = 0;
        for (int64_t idx = 0; idx < nk; idx++) {
            int64_t rem = idx;
            double r = 0.0;
            for (int t = d - 1; t >= 0; t--) {
                int64_t k_t = rem % N[t] - N[t] / 2;
                rem /= N[t];
                r += reduced_product(k_t, x[j * d + t]);
            }
            double ph = 2.0 * ORA_PI * r;
            acc += fhat[idx] * (cos(ph) - I * sin(ph));
        }
        f[j] = acc;
    }
}

/* hhat_k = sum_{j=0}^{M-1} f_j e^{+2 pi i k.x_j},  k in I_N   (Section 1, adjoint sum). */
void ora_ndft_adjoint(int d, const int64_t *N, int64_t M, const double *x, const cplx *f,
                      cplx *fhat)
{
    const int64_t nk = prod64(d, N);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t idx = 0; idx < nk; idx++) {
        int64_t k[3] = {0, 0, 0};
        int64_t rem = idx;
        for (int t = d - 1; t >= 0; t--) {
            k[t] = rem % N[t] - N[t] / 2;
            rem /= N[t];
        }
        cplx acc = 0;
        for (int64_t j = 0; j < M; j++) {
            double r = 0.0;
            for (int t = 0; t < d; t++) r += reduced_product(k[t], x[j * d + t]);
            double ph = 2.0 * ORA_PI * r;
            acc += f[j] * (cos(ph) + I * sin(ph));
        }
        fhat[idx] = acc;
    }
}

/* The one-dimensional factors of the NDFT's exponential on every axis of one node: since
 * e^{sign 2 pi i k.x} = prod_t e^{sign 2 pi i k_t x_t}, row t of E (N_t values, position
 * k_t + N_t/2) holds e^{sign 2 pi i k_t x_t}, each evaluated with the exact phase reduction. */
static void axis_factors(int d, const int64_t *N, const double *xj, int sign, cplx *E)
{
    int64_t off = 0;
    for (int t = 0; t < d; t++) {
        for (int64_t i = 0; i < N[t]; i++) {
            double ph = 2.0 * ORA_PI * reduced_product(i - N[t] / 2, xj[t]);
            E[off + i] = cos(ph) + sign * I * sin(ph);
        }
        off += N[t];
    }
}

/* The NDFT of Section 1 (eq. NDFT), f_j = sum_{k in I_N} fhat_k e^{-2 pi i k.x_j}, with each
 * term's exponential formed as the product of its per-axis factors (axis_factors) instead of
 * one cosine and sine of the summed phase. Same sum in the same order as ora_ndft; only the
 * rounding of the exponentials differs. */
void ora_ndft_tab(int d, const int64_t *N, int64_t M, const double *x, const cplx *fhat,
                  cplx *f)
{
    const int64_t nk = prod64(d, N);
    int64_t tot = 0;
    for (int t = 0; t < d; t++) tot += N[t];
#pragma omp parallel
    {
        cplx *E = (cplx *)malloc((size_t)tot * sizeof(cplx));
#pragma omp for schedule(dynamic, 4)
        for (int64_t j = 0; j < M; j++) {
            axis_factors(d, N, x + j * d, -1, E);
            cplx acc = 0;
            for (int64_t idx = 0; idx < nk; idx++) {
                int64_t rem = idx, off = 0, kk[3] = {0, 0, 0};
                for (int t = d - 1; t >= 0; t--) {
                    kk[t] = rem % N[t];
                    rem /= N[t];
                }
                cplx e = 1.0;
                for (int t = 0; t < d; t++) {
                    e *= E[off + kk[t]];
                    off += N[t];
                }
                acc += fhat[idx] * e;
            }
            f[j] = acc;
        }
        free(E);
    }
}

/* The adjoint NDFT of Section 1 at the K listed coefficients only:
 * out[q] = sum_{j=0}^{M-1} f_j e^{+2 pi i k.x_j}, k the multi-index at row-major position
 * kidx[q] of I_N (axis t at k_t + N_t/2). Exponentials as in ora_ndft_tab. The sum over j is
 * split into contiguous node ranges, one per thread, whose partial sums are added in range
 * order (the same sum as ora_ndft_adjoint up to rounding order). */
void ora_ndft_adjoint_at(int d, const int64_t *N, int64_t M, const double *x, const cplx *f,
                         int64_t K, const int64_t *kidx, cplx *out)
{
    int64_t tot = 0;
    for (int t = 0; t < d; t++) tot += N[t];
    int64_t *pos = (int64_t *)malloc((size_t)(K > 0 ? K : 1) * 3 * sizeof(int64_t));
    for (int64_t q = 0; q < K; q++) {
        int64_t rem = kidx[q], off = tot;
        for (int t = d - 1; t >= 0; t--) {
            off -= N[t];
            pos[q * 3 + t] = off + rem % N[t];  /* position of k_t's factor in E */
            rem /= N[t];
        }
    }
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    cplx *part = (cplx *)calloc((size_t)nth * (size_t)(K > 0 ? K : 1), sizeof(cplx));
#pragma omp parallel num_threads(nth)
    {
        int me = 0, nt = 1;
#ifdef _OPENMP
        me = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        const int64_t j0 = M * me / nt, j1 = M * (me + 1) / nt;
        cplx *E = (cplx *)malloc((size_t)tot * sizeof(cplx));
        cplx *acc = part + (size_t)me * (size_t)K;
        for (int64_t j = j0; j < j1; j++) {
            axis_factors(d, N, x + j * d, +1, E);
            for (int64_t q = 0; q < K; q++) {
                cplx e = 1.0;
                for (int t = 0; t < d; t++) e *= E[pos[q * 3 + t]];
                acc[q] += f[j] * e;
            }
        }
        free(E);
    }
    for (int64_t q = 0; q < K; q++) {
        cplx s = 0;
        for (int r = 0; r < nth; r++) s += part[(size_t)r * (size_t)K + q];
        out[q] = s;
    }
    free(part);
    free(pos);
}

/* Partial derivatives of the trigonometric polynomial (Section 2, eq. trigpoly):
 * df[j*d + t] = d f / d x_t (x_j) = sum_k (-2 pi i k_t) fhat_k e^{-2 pi i k.x_j}. */
void ora_ndft_grad(int d, const int64_t *N, int64_t M, const double *x, const cplx *fhat,
                   cplx *df)
{
    const int64_t nk = prod64(d, N);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < M; j++) {
        cplx acc[3] = {0, 0, 0};
        for (int64_t idx = 0; idx < nk; idx++) {
            int64_t k[3] = {0, 0, 0};
            int64_t rem = idx;
            double r = 0.0;
            for (int t = d - 1; t >= 0; t--) {
                k[t] = rem % N[t] - N[t] / 2;
                rem /= N[t];
                r += reduced_product(k[t], x[j * d + t]);
            }
            double ph = 2.0 * ORA_PI * r;
            cplx term = fhat[idx] * (cos(ph) - I * sin(ph));
            for (int t = 0; t < d; t++) acc[t] += (-2.0 * ORA_PI * I * (double)k[t]) * term;
        }
        for (int t = 0; t < d; t++) df[j * d + t] = acc[t];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Kaiser-Bessel window (Section 2, eq. window and eq. window_cutoff; formula: see header)     */
/* ------------------------------------------------------------------------------------------ */

/* Modified Bessel function of the first kind, order 0, from its power series
 * I0(z) = sum_{j>=0} (z^2/4)^j / (j!)^2 (all terms positive: no cancellation). */
double ora_bessel_i0(double z)
{
    const double q = 0.25 * z * z;
    double term = 1.0, sum = 1.0;
    for (int j = 1; j < 1000; j++) {
        term *= q / ((double)j * (double)j);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* Shape parameter b = pi (2 - 1/sigma) with sigma = n / N. */
double ora_kb_b(int64_t n, int64_t N)
{
    const double sigma = (double)n / (double)N;
    return ORA_PI * (2.0 - 1.0 / sigma);
}

/* Truncated window in grid units, psi(t) = phi(t / n) for |t| <= m and 0 otherwise
 * (eq. window_cutoff). At |t| = m the value is the limit b / pi. */
double ora_kb_psi(double t, int m, double b)
{
    const double s = (double)m * (double)m - t * t;
    if (s < 0.0) return 0.0;
    const double u = sqrt(s);
    if (u == 0.0) return b / ORA_PI;
    return sinh(b * u) / (ORA_PI * u);
}

/* d psi / d t inside the support: with u = sqrt(m^2 - t^2),
 * psi'(t) = -t (b u cosh(b u) - sinh(b u)) / (pi u^3); for small b u the bracket divided by
 * u^3 is replaced by its Taylor series b^3/3 (1 + z^2/10 + z^4/280), z = b u. */
double ora_kb_dpsi(double t, int m, double b)
{
    const double s = (double)m * (double)m - t * t;
    if (s < 0.0) return 0.0;
    const double u = sqrt(s);
    const double z = b * u;
    double g;
    if (z < 1e-2) {
        g = b * b * b / 3.0 * (1.0 + z * z / 10.0 + z * z * z * z / 280.0);
    } else {
        g = (z * cosh(z) - sinh(z)) / (u * u * u);
    }
    return -t * g / ORA_PI;
}

/* Fourier transform of the (untruncated) window at integer frequency k: the Fourier
 * coefficient c_k of the 1-periodised window (Section 2, c_k = phihat(k)). */
double ora_kb_phihat(int64_t k, int64_t n, int m, double b)
{
    const double w = 2.0 * ORA_PI * (double)k / (double)n;
    const double s = b * b - w * w;
    if (s < 0.0) return 0.0;
    return ora_bessel_i0((double)m * sqrt(s)) / (double)n;
}

/* ------------------------------------------------------------------------------------------ */
/* The other windows the paper names (Section 4.1: Gaussian, B-spline, sinc); their formulas are */
/* the standard Fourier pairs (the paper defers them to Plonka-Potts-Steidl-Tasche, Ch. 7.2).    */
/* All in grid units t = n x; each pair satisfies phihat(k) = (1/n) * FT[psi](k / n), where     */
/* FT[psi](nu) = int psi(t) e^{-2 pi i nu t} dt.                                                */
/* ------------------------------------------------------------------------------------------ */

enum { ORA_KB = 0, ORA_GAUSS = 1, ORA_BSPLINE = 2, ORA_SINC = 3 };

/* Centred cardinal B-spline of order p (support [-p/2, p/2]) by the recursion
 * M_p(t) = ((p/2 + t) M_{p-1}(t + 1/2) + (p/2 - t) M_{p-1}(t - 1/2)) / (p - 1), M_1 = 1 on
 * [-1/2, 1/2) (all terms non-negative). */
double ora_bspline(int p, double t)
{
    if (p == 1) return (t >= -0.5 && t < 0.5) ? 1.0 : 0.0;
    if (t <= -0.5 * p || t >= 0.5 * p) return 0.0;
    return ((0.5 * p + t) * ora_bspline(p - 1, t + 0.5) + (0.5 * p - t) * ora_bspline(p - 1, t - 0.5)) /
           (double)(p - 1);
}

static double ora_sinc(double u) { return u == 0.0 ? 1.0 : sin(u) / u; }

/* Shape parameter of window w on an axis with FFT length n and bandwidth N:
 * KB: b = pi (2 - 1/sigma); Gaussian: b = 2 sigma m / ((2 sigma - 1) pi);
 * sinc: a = (2 sigma - 1) / (2 m sigma); B-spline: unused. */
double ora_window_param(int w, int64_t n, int64_t N, int m)
{
    w &= 0xff; /* window kind (the lookup-table setting does not change the pair) */
    const double sigma = (double)n / (double)N;
    switch (w) {
    case ORA_GAUSS: return 2.0 * sigma * m / ((2.0 * sigma - 1.0) * ORA_PI);
    case ORA_SINC: return (2.0 * sigma - 1.0) / (2.0 * m * sigma);
    case ORA_BSPLINE: return 0.0;
    default: return ora_kb_b(n, N);
    }
}

/* Truncated window psi(t) (0 for |t| > m). Gaussian: e^{-t^2/b}; B-spline: M_{2m}(t);
 * sinc: sinc^{2m}(pi a t); KB: see ora_kb_psi. */
double ora_window_psi(int w, double t, int m, double prm)
{
    w &= 0xff; /* window kind (the lookup-table setting does not change the pair) */
    if (fabs(t) > (double)m) return 0.0;
    switch (w) {
    case ORA_GAUSS: return exp(-t * t / prm);
    case ORA_BSPLINE: return ora_bspline(2 * m, t);
    case ORA_SINC: return pow(ora_sinc(ORA_PI * prm * t), 2 * m);
    default: return ora_kb_psi(t, m, prm);
    }
}

/* d psi / d t inside the support. */
double ora_window_dpsi(int w, double t, int m, double prm)
{
    w &= 0xff; /* window kind (the lookup-table setting does not change the pair) */
    if (fabs(t) > (double)m) return 0.0;
    switch (w) {
    case ORA_GAUSS: return -2.0 * t / prm * exp(-t * t / prm);
    case ORA_BSPLINE: return ora_bspline(2 * m - 1, t + 0.5) - ora_bspline(2 * m - 1, t - 0.5);
    case ORA_SINC: {
        const double u = ORA_PI * prm * t;
        if (u == 0.0) return 0.0;
        const double ds = (u * cos(u) - sin(u)) / (u * u);  /* d sinc / du */
        return 2.0 * m * pow(ora_sinc(u), 2 * m - 1) * ds * ORA_PI * prm;
    }
    default: return ora_kb_dpsi(t, m, prm);
    }
}

/* PRE_LIN_PSI (Section 3.1, Table tab:nfftflags): psi read from a table of its values at the
 * K points per unit t = j / K, linearly interpolated. A window spec w carries the window kind
 * in its low 8 bits and K in the bits above (K = 0: the exact window). The interpolant between
 * samples j / K and (j + 1) / K of |t| is written out directly (the samples are the table). */
double ora_window_psi_eval(int w, double t, int m, double prm)
{
    const int K = w >> 8;
    if (K == 0) return ora_window_psi(w, t, m, prm);
    const double a = fabs(t);
    if (a > (double)m) return 0.0;
    const double u = a * (double)K;
    const double j = floor(u), lam = u - j;
    return (1.0 - lam) * ora_window_psi(w, j / K, m, prm) +
           lam * ora_window_psi(w, (j + 1.0) / K, m, prm);
}

/* d/dt of the interpolant: the slope of the segment holding |t|, times sign(t). At a sample
 * point (a kink) this is the right derivative in t, the limit from larger t: the segment above
 * |t| for t >= 0, the one below |t| for t < 0; at t = +m, where the cut-off window jumps to 0,
 * it is the derivative from inside the support, as for the exact window. */
double ora_window_dpsi_eval(int w, double t, int m, double prm)
{
    const int K = w >> 8;
    if (K == 0) return ora_window_dpsi(w, t, m, prm);
    const double a = fabs(t);
    if (a > (double)m) return 0.0;
    double j = t >= 0 ? floor(a * (double)K) : ceil(a * (double)K) - 1.0;
    if (j > (double)m * K - 1.0) j = (double)m * K - 1.0;
    const double slope =
        (ora_window_psi(w, (j + 1.0) / K, m, prm) - ora_window_psi(w, j / K, m, prm)) * K;
    return t < 0 ? -slope : slope;
}

/* phihat(k) = (1/n) FT[psi_untruncated](k/n). Gaussian: sqrt(pi b) e^{-b (pi k/n)^2} / n;
 * B-spline: sinc^{2m}(pi k / n) / n; sinc: M_{2m}(k / (n a)) / (n a); KB: ora_kb_phihat. */
double ora_window_phihat(int w, int64_t k, int64_t n, int m, double prm)
{
    w &= 0xff; /* window kind (the lookup-table setting does not change the pair) */
    const double nu = (double)k / (double)n;
    switch (w) {
    case ORA_GAUSS: return sqrt(ORA_PI * prm) * exp(-prm * ORA_PI * ORA_PI * nu * nu) / (double)n;
    case ORA_BSPLINE: return pow(ora_sinc(ORA_PI * nu), 2 * m) / (double)n;
    case ORA_SINC: return ora_bspline(2 * m, nu / prm) / (prm * (double)n);
    default: return ora_kb_phihat(k, n, m, prm);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* FFT (Algorithm "NFFT", d-variate FFT step)                                                  */
/* ------------------------------------------------------------------------------------------ */

/* Unnormalised 1-D DFT a_l <- sum_k a_k e^{sign 2 pi i k l / n}, in place.
 * Even n: split into even and odd samples (radix 2, recursively); odd n: direct sum. */
static void fft1(cplx *a, int64_t n, int sign, cplx *scratch)
{
    if (n == 1) return;
    if (n % 2 != 0) {
        for (int64_t l = 0; l < n; l++) {
            cplx acc = 0;
            for (int64_t k = 0; k < n; k++) {
                double ph = 2.0 * ORA_PI * (double)((k * l) % n) / (double)n;
                acc += a[k] * (cos(ph) + sign * I * sin(ph));
            }
            scratch[l] = acc;
        }
        memcpy(a, scratch, (size_t)n * sizeof(cplx));
        return;
    }
    const int64_t h = n / 2;
    for (int64_t i = 0; i < h; i++) {
        scratch[i] = a[2 * i];
        scratch[h + i] = a[2 * i + 1];
    }
    fft1(scratch, h, sign, a);
    fft1(scratch + h, h, sign, a);
    for (int64_t k = 0; k < h; k++) {
        double ph = 2.0 * ORA_PI * (double)k / (double)n;
        cplx w = cos(ph) + sign * I * sin(ph);
        cplx e = scratch[k];
        cplx o = w * scratch[h + k];
        a[k] = e + o;
        a[k + h] = e - o;
    }
}

/* d-variate unnormalised DFT of a row-major n[0] x ... x n[d-1] array, in place:
 * a_l <- sum_k a_k e^{sign 2 pi i k.(l / n)} (sign = -1: forward, +1: inverse). */
void ora_fft(int d, const int64_t *n, cplx *a, int sign)
{
    for (int t = 0; t < d; t++) {
        int64_t inner = 1, outer = 1;
        for (int u = t + 1; u < d; u++) inner *= n[u];
        for (int u = 0; u < t; u++) outer *= n[u];
        const int64_t len = n[t];
        const int64_t lines = outer * inner;
#pragma omp parallel
        {
            cplx *line = (cplx *)malloc((size_t)len * sizeof(cplx));
            cplx *scr = (cplx *)malloc((size_t)len * sizeof(cplx));
#pragma omp for schedule(static)
            for (int64_t q = 0; q < lines; q++) {
                const int64_t o = q / inner, i = q % inner;
                const int64_t base = o * len * inner + i;
                for (int64_t p = 0; p < len; p++) line[p] = a[base + p * inner];
                fft1(line, len, sign, scr);
                for (int64_t p = 0; p < len; p++) a[base + p * inner] = line[p];
            }
            free(line);
            free(scr);
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* The three steps of Algorithm "NFFT" and of Algorithm "adjoint NFFT"                         */
/* ------------------------------------------------------------------------------------------ */

/* Product over the axes of the Fourier coefficients c_k = phihat_t(k_t) of window w. */
static double phihat_prod(int w, int d, const int64_t *k, const int64_t *N, const int64_t *n, int m)
{
    double c = 1.0;
    for (int t = 0; t < d; t++)
        c *= ora_window_phihat(w, k[t], n[t], m, ora_window_param(w, n[t], N[t], m));
    return c;
}

/* Step D (Algorithm "NFFT", first loop; Section 2, choice of ghat):
 * ghat_{k mod n} = fhat_k / (|I_n| c_k) for k in I_N, and 0 on I_n \ I_N. */
void ora_nfft_D_w(int w, int d, const int64_t *N, const int64_t *n, int m, const cplx *fhat,
                  cplx *ghat)
{
    const int64_t nk = prod64(d, N), ng = prod64(d, n);
    memset(ghat, 0, (size_t)ng * sizeof(cplx));
    for (int64_t idx = 0; idx < nk; idx++) {
        int64_t k[3] = {0, 0, 0};
        int64_t rem = idx;
        for (int t = d - 1; t >= 0; t--) {
            k[t] = rem % N[t] - N[t] / 2;
            rem /= N[t];
        }
        int64_t g = 0;
        for (int t = 0; t < d; t++) g = g * n[t] + mod64(k[t], n[t]);
        ghat[g] = fhat[idx] / ((double)ng * phihat_prod(w, d, k, N, n, m));
    }
}

void ora_nfft_D(int d, const int64_t *N, const int64_t *n, int m, const cplx *fhat, cplx *ghat)
{
    ora_nfft_D_w(ORA_KB, d, N, n, m, fhat, ghat);
}

/* Step D^H (Algorithm "adjoint NFFT", last loop):
 * hhat_k = ghat_{k mod n} / (|I_n| c_k) for k in I_N. */
void ora_nfft_DH_w(int w, int d, const int64_t *N, const int64_t *n, int m, const cplx *ghat,
                   cplx *fhat)
{
    const int64_t nk = prod64(d, N), ng = prod64(d, n);
    for (int64_t idx = 0; idx < nk; idx++) {
        int64_t k[3] = {0, 0, 0};
        int64_t rem = idx;
        for (int t = d - 1; t >= 0; t--) {
            k[t] = rem % N[t] - N[t] / 2;
            rem /= N[t];
        }
        int64_t g = 0;
        for (int t = 0; t < d; t++) g = g * n[t] + mod64(k[t], n[t]);
        fhat[idx] = ghat[g] / ((double)ng * phihat_prod(w, d, k, N, n, m));
    }
}

void ora_nfft_DH(int d, const int64_t *N, const int64_t *n, int m, const cplx *ghat, cplx *fhat)
{
    ora_nfft_DH_w(ORA_KB, d, N, n, m, ghat, fhat);
}

/* The box of grid indices I_{n,m}(x_j) of eq. Inm: for each axis, the integers l with
 * n x - m <= l <= n x + m (closed interval). */
static void support_box(int d, const int64_t *n, int m, const double *xj, double *nx, int64_t *lo,
                        int64_t *hi)
{
    for (int t = 0; t < d; t++) {
        nx[t] = (double)n[t] * xj[t];
        lo[t] = (int64_t)ceil(nx[t] - (double)m);
        hi[t] = (int64_t)floor(nx[t] + (double)m);
    }
}

/* Step B (Algorithm "NFFT", last loop; eq. s_approx):
 * f_j = sum_{l in I_{n,m}(x_j)} g_{l mod n} psi~(x_j - l/n), with the tensor-product window
 * psi~(y) = prod_t psi_t(n_t y_t). */
void ora_nfft_B_w(int w, int d, const int64_t *N, const int64_t *n, int m, int64_t M,
                  const double *x,
                const cplx *g, cplx *f)
{
    double b[3] = {0, 0, 0};
    for (int t = 0; t < d; t++) b[t] = ora_window_param(w, n[t], N[t], m);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; j++) {
        double nx[3];
        int64_t lo[3], hi[3], l[3];
        support_box(d, n, m, x + j * d, nx, lo, hi);
        for (int t = 0; t < d; t++) l[t] = lo[t];
        cplx acc = 0;
        for (;;) {
            double wt = 1.0;
            int64_t gi = 0;
            for (int t = 0; t < d; t++) {
                wt *= ora_window_psi_eval(w, nx[t] - (double)l[t], m, b[t]);
                gi = gi * n[t] + mod64(l[t], n[t]);
            }
            acc += g[gi] * wt;
            int t = d - 1;
            while (t >= 0 && l[t] == hi[t]) {
                l[t] = lo[t];
                t--;
            }
            if (t < 0) break;
            l[t]++;
        }
        f[j] = acc;
    }
}

/* Step B^H (Algorithm "adjoint NFFT", first loop):
 * g_l = sum_{j in I^T_{n,m}(l)} f_j psi~(x_j - l/n); evaluated node by node. The grid is split
 * into slabs of consecutive indices l_0 on the first axis, one slab per thread; every thread
 * visits all nodes in order and adds only the taps in its own slab, so every g_l receives its
 * terms in node order, exactly as a single thread would add them. */
void ora_nfft_BH_w(int w, int d, const int64_t *N, const int64_t *n, int m, int64_t M,
                  const double *x,
                 const cplx *f, cplx *g)
{
    double b[3] = {0, 0, 0};
    for (int t = 0; t < d; t++) b[t] = ora_window_param(w, n[t], N[t], m);
    memset(g, 0, (size_t)prod64(d, n) * sizeof(cplx));
#pragma omp parallel
    {
        int me = 0, nt = 1;
#ifdef _OPENMP
        me = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        const int64_t s0 = n[0] * me / nt, s1 = n[0] * (me + 1) / nt;  /* rows [s0, s1) */
        for (int64_t j = 0; j < M; j++) {
            double nx[3];
            int64_t lo[3], hi[3], l[3];
            support_box(d, n, m, x + j * d, nx, lo, hi);
            int mine = 0;
            for (int64_t l0 = lo[0]; l0 <= hi[0]; l0++) {
                const int64_t r = mod64(l0, n[0]);
                if (r >= s0 && r < s1) mine = 1;
            }
            if (!mine) continue;
            for (int t = 0; t < d; t++) l[t] = lo[t];
            for (;;) {
                const int64_t r0 = mod64(l[0], n[0]);
                if (r0 >= s0 && r0 < s1) {
                    double wt = 1.0;
                    int64_t gi = 0;
                    for (int t = 0; t < d; t++) {
                        wt *= ora_window_psi_eval(w, nx[t] - (double)l[t], m, b[t]);
                        gi = gi * n[t] + mod64(l[t], n[t]);
                    }
                    g[gi] += f[j] * wt;
                }
                int t = d - 1;
                while (t >= 0 && l[t] == hi[t]) {
                    l[t] = lo[t];
                    t--;
                }
                if (t < 0) break;
                l[t]++;
            }
        }
    }
}

/* Derivative of the approximation s of eq. s_approx with respect to the node coordinates:
 * ds[j*d + t] = d s / d x_t (x_j) = sum_{l} g_{l mod n} n_t psi_t'(n_t x_t - l_t)
 *               prod_{u != t} psi_u(n_u x_u - l_u), over the same support box. */
void ora_nfft_dB_w(int w, int d, const int64_t *N, const int64_t *n, int m, int64_t M,
                  const double *x,
                 const cplx *g, cplx *ds)
{
    double b[3] = {0, 0, 0};
    for (int t = 0; t < d; t++) b[t] = ora_window_param(w, n[t], N[t], m);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; j++) {
        double nx[3];
        int64_t lo[3], hi[3], l[3];
        support_box(d, n, m, x + j * d, nx, lo, hi);
        for (int t = 0; t < d; t++) l[t] = lo[t];
        cplx acc[3] = {0, 0, 0};
        for (;;) {
            double wv[3], dw[3];
            int64_t gi = 0;
            for (int t = 0; t < d; t++) {
                wv[t] = ora_window_psi_eval(w, nx[t] - (double)l[t], m, b[t]);
                dw[t] = (double)n[t] * ora_window_dpsi_eval(w, nx[t] - (double)l[t], m, b[t]);
                gi = gi * n[t] + mod64(l[t], n[t]);
            }
            for (int t = 0; t < d; t++) {
                double p = dw[t];
                for (int u = 0; u < d; u++)
                    if (u != t) p *= wv[u];
                acc[t] += g[gi] * p;
            }
            int t = d - 1;
            while (t >= 0 && l[t] == hi[t]) {
                l[t] = lo[t];
                t--;
            }
            if (t < 0) break;
            l[t]++;
        }
        for (int t = 0; t < d; t++) ds[j * d + t] = acc[t];
    }
}


void ora_nfft_B(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
                const cplx *g, cplx *f)
{
    ora_nfft_B_w(ORA_KB, d, N, n, m, M, x, g, f);
}

void ora_nfft_BH(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
                 const cplx *f, cplx *g)
{
    ora_nfft_BH_w(ORA_KB, d, N, n, m, M, x, f, g);
}

void ora_nfft_dB(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
                 const cplx *g, cplx *ds)
{
    ora_nfft_dB_w(ORA_KB, d, N, n, m, M, x, g, ds);
}

/* ------------------------------------------------------------------------------------------ */
/* Whole transforms                                                                           */
/* ------------------------------------------------------------------------------------------ */

/* Algorithm "NFFT": D, then the forward d-variate FFT, then B (window w). */
int ora_nfft_w(int w, int d, const int64_t *N, const int64_t *n, int m, int64_t M,
               const double *x, const cplx *fhat, cplx *f)
{
    cplx *g = (cplx *)malloc((size_t)prod64(d, n) * sizeof(cplx));
    if (!g) return 1;
    ora_nfft_D_w(w, d, N, n, m, fhat, g);
    ora_fft(d, n, g, -1);
    ora_nfft_B_w(w, d, N, n, m, M, x, g, f);
    free(g);
    return 0;
}

int ora_nfft(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
             const cplx *fhat, cplx *f)
{
    return ora_nfft_w(ORA_KB, d, N, n, m, M, x, fhat, f);
}

/* Algorithm "adjoint NFFT": B^H, then the inverse (sign +1) d-variate FFT, then D^H. */
int ora_nfft_adjoint_w(int w, int d, const int64_t *N, const int64_t *n, int m, int64_t M,
                       const double *x, const cplx *f, cplx *fhat)
{
    cplx *g = (cplx *)malloc((size_t)prod64(d, n) * sizeof(cplx));
    if (!g) return 1;
    ora_nfft_BH_w(w, d, N, n, m, M, x, f, g);
    ora_fft(d, n, g, +1);
    ora_nfft_DH_w(w, d, N, n, m, g, fhat);
    free(g);
    return 0;
}

int ora_nfft_adjoint(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
                     const cplx *f, cplx *fhat)
{
    return ora_nfft_adjoint_w(ORA_KB, d, N, n, m, M, x, f, fhat);
}

/* Node gradient of a real loss through the NFFT (PyTorch's conjugate-Wirtinger convention):
 * gx[j*d + t] = Re( conj(w_j) * d s_c / d x_t (x_j) ), where s_c is the NFFT approximation
 * built from the coefficients c (steps D and F), and w is the upstream weight per node.
 * For the forward transform c = fhat and w = grad f; for the adjoint c = grad hhat and w = f. */
int ora_nfft_grad_x_w(int win, int d, const int64_t *N, const int64_t *n, int m, int64_t M,
                      const double *x, const cplx *c, const cplx *w, double *gx)
{
    cplx *g = (cplx *)malloc((size_t)prod64(d, n) * sizeof(cplx));
    cplx *ds = (cplx *)malloc((size_t)(M > 0 ? M : 1) * d * sizeof(cplx));
    if (!g || !ds) {
        free(g);
        free(ds);
        return 1;
    }
    ora_nfft_D_w(win, d, N, n, m, c, g);
    ora_fft(d, n, g, -1);
    ora_nfft_dB_w(win, d, N, n, m, M, x, g, ds);
    for (int64_t j = 0; j < M; j++)
        for (int t = 0; t < d; t++) gx[j * d + t] = creal(conj(w[j]) * ds[j * d + t]);
    free(g);
    free(ds);
    return 0;
}

int ora_nfft_grad_x(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
                    const cplx *c, const cplx *w, double *gx)
{
    return ora_nfft_grad_x_w(ORA_KB, d, N, n, m, M, x, c, w, gx);
}
