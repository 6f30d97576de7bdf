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

/* Product over the axes of the Fourier coefficients c_k = phihat_t(k_t) of the window. */
static double phihat_prod(int d, const int64_t *k, const int64_t *N, const int64_t *n, int m)
{
    double c = 1.0;
    for (int t = 0; t < d; t++) c *= ora_kb_phihat(k[t], n[t], m, ora_kb_b(n[t], N[t]));
    return c;
}

/* Step D (Algorithm "NFFT", first loop; Section 2, choice of ghat):
 * ghat_{k mod n} = fhat_k / (|I_n| c_k) for k in I_N, and 0 on I_n \ I_N. */
void ora_nfft_D(int d, const int64_t *N, const int64_t *n, int m, const cplx *fhat, cplx *ghat)
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
        ghat[g] = fhat[idx] / ((double)ng * phihat_prod(d, k, N, n, m));
    }
}

/* Step D^H (Algorithm "adjoint NFFT", last loop):
 * hhat_k = ghat_{k mod n} / (|I_n| c_k) for k in I_N. */
void ora_nfft_DH(int d, const int64_t *N, const int64_t *n, int m, const cplx *ghat, cplx *fhat)
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
        fhat[idx] = ghat[g] / ((double)ng * phihat_prod(d, k, N, n, m));
    }
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
void ora_nfft_B(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
                const cplx *g, cplx *f)
{
    double b[3] = {0, 0, 0};
    for (int t = 0; t < d; t++) b[t] = ora_kb_b(n[t], N[t]);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; j++) {
        double nx[3];
        int64_t lo[3], hi[3], l[3];
        support_box(d, n, m, x + j * d, nx, lo, hi);
        for (int t = 0; t < d; t++) l[t] = lo[t];
        cplx acc = 0;
        for (;;) {
            double w = 1.0;
            int64_t gi = 0;
            for (int t = 0; t < d; t++) {
                w *= ora_kb_psi(nx[t] - (double)l[t], m, b[t]);
                gi = gi * n[t] + mod64(l[t], n[t]);
            }
            acc += g[gi] * w;
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
 * g_l = sum_{j in I^T_{n,m}(l)} f_j psi~(x_j - l/n); evaluated node by node. */
void ora_nfft_BH(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
                 const cplx *f, cplx *g)
{
    double b[3] = {0, 0, 0};
    for (int t = 0; t < d; t++) b[t] = ora_kb_b(n[t], N[t]);
    memset(g, 0, (size_t)prod64(d, n) * sizeof(cplx));
    for (int64_t j = 0; j < M; j++) {
        double nx[3];
        int64_t lo[3], hi[3], l[3];
        support_box(d, n, m, x + j * d, nx, lo, hi);
        for (int t = 0; t < d; t++) l[t] = lo[t];
        for (;;) {
            double w = 1.0;
            int64_t gi = 0;
            for (int t = 0; t < d; t++) {
                w *= ora_kb_psi(nx[t] - (double)l[t], m, b[t]);
                gi = gi * n[t] + mod64(l[t], n[t]);
            }
            g[gi] += f[j] * w;
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

/* Derivative of the approximation s of eq. s_approx with respect to the node coordinates:
 * ds[j*d + t] = d s / d x_t (x_j) = sum_{l} g_{l mod n} n_t psi_t'(n_t x_t - l_t)
 *               prod_{u != t} psi_u(n_u x_u - l_u), over the same support box. */
void ora_nfft_dB(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
                 const cplx *g, cplx *ds)
{
    double b[3] = {0, 0, 0};
    for (int t = 0; t < d; t++) b[t] = ora_kb_b(n[t], N[t]);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; j++) {
        double nx[3];
        int64_t lo[3], hi[3], l[3];
        support_box(d, n, m, x + j * d, nx, lo, hi);
        for (int t = 0; t < d; t++) l[t] = lo[t];
        cplx acc[3] = {0, 0, 0};
        for (;;) {
            double w[3], dw[3];
            int64_t gi = 0;
            for (int t = 0; t < d; t++) {
                w[t] = ora_kb_psi(nx[t] - (double)l[t], m, b[t]);
                dw[t] = (double)n[t] * ora_kb_dpsi(nx[t] - (double)l[t], m, b[t]);
                gi = gi * n[t] + mod64(l[t], n[t]);
            }
            for (int t = 0; t < d; t++) {
                double p = dw[t];
                for (int u = 0; u < d; u++)
                    if (u != t) p *= w[u];
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

/* ------------------------------------------------------------------------------------------ */
/* Whole transforms                                                                           */
/* ------------------------------------------------------------------------------------------ */

/* Algorithm "NFFT": D, then the forward d-variate FFT, then B. */
int ora_nfft(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
             const cplx *fhat, cplx *f)
{
    cplx *g = (cplx *)malloc((size_t)prod64(d, n) * sizeof(cplx));
    if (!g) return 1;
    ora_nfft_D(d, N, n, m, fhat, g);
    ora_fft(d, n, g, -1);
    ora_nfft_B(d, N, n, m, M, x, g, f);
    free(g);
    return 0;
}

/* Algorithm "adjoint NFFT": B^H, then the inverse (sign +1) d-variate FFT, then D^H. */
int ora_nfft_adjoint(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
                     const cplx *f, cplx *fhat)
{
    cplx *g = (cplx *)malloc((size_t)prod64(d, n) * sizeof(cplx));
    if (!g) return 1;
    ora_nfft_BH(d, N, n, m, M, x, f, g);
    ora_fft(d, n, g, +1);
    ora_nfft_DH(d, N, n, m, g, fhat);
    free(g);
    return 0;
}

/* Node gradient of a real loss through the NFFT (PyTorch's conjugate-Wirtinger convention):
 * gx[j*d + t] = Re( conj(w_j) * d s_c / d x_t (x_j) ), where s_c is the NFFT approximation
 * built from the coefficients c (steps D and F), and w is the upstream weight per node.
 * For the forward transform c = fhat and w = grad f; for the adjoint c = grad hhat and w = f. */
int ora_nfft_grad_x(int d, const int64_t *N, const int64_t *n, int m, int64_t M, const double *x,
                    const cplx *c, const cplx *w, double *gx)
{
    cplx *g = (cplx *)malloc((size_t)prod64(d, n) * sizeof(cplx));
    cplx *ds = (cplx *)malloc((size_t)(M > 0 ? M : 1) * d * sizeof(cplx));
    if (!g || !ds) {
        free(g);
        free(ds);
        return 1;
    }
    ora_nfft_D(d, N, n, m, c, g);
    ora_fft(d, n, g, -1);
    ora_nfft_dB(d, N, n, m, M, x, g, ds);
    for (int64_t j = 0; j < M; j++)
        for (int t = 0; t < d; t++) gx[j * d + t] = creal(conj(w[j]) * ds[j * d + t]);
    free(g);
    free(ds);
    return 0;
}
