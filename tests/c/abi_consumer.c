/* A plain C consumer of the library's C ABI (include/gbnfft.h): no Python, no PyTorch.
 * Creates a 2-D FP64 plan (N = 16 x 12, n = 32 x 24, m = 6), transfers nodes and coefficients
 * through the host-buffer entry points, and checks the forward NFFT against a direct NDFT
 * f_j = sum_k fhat_k e^{-2 pi i k.x_j} (Section 2, eq. NDFT) and the adjoint against
 * hhat_k = sum_j f_j e^{+2 pi i k.x_j}. Prints "max_rel_fwd max_rel_adj" and exits 0 when both
 * are below 1e-9 (the window error at m = 6, sigma = 2 is ~1e-11). */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "gbnfft.h"

#define N0 16
#define N1 12
#define M 200

static double lcg(uint64_t *s)
{
    *s = *s * 6364136223846793005ULL + 1442695040888963407ULL;
    return (double)(*s >> 11) / 9007199254740992.0; /* [0, 1) */
}

int main(void)
{
    const double pi = 3.14159265358979323846;
    const int64_t N[2] = {N0, N1}, n[2] = {32, 24};
    double *x = malloc(sizeof(double) * 2 * M);
    double *fhat = malloc(sizeof(double) * 2 * N0 * N1); /* interleaved complex */
    double *f = malloc(sizeof(double) * 2 * M);
    double *hh = malloc(sizeof(double) * 2 * N0 * N1);
    double *fv = malloc(sizeof(double) * 2 * M);
    uint64_t seed = 1810;
    for (int j = 0; j < 2 * M; j++) x[j] = lcg(&seed) - 0.5;
    for (int k = 0; k < 2 * N0 * N1; k++) fhat[k] = lcg(&seed) - 0.5;
    for (int j = 0; j < 2 * M; j++) fv[j] = lcg(&seed) - 0.5;

    nfft_plan p = NULL;
    int rc = nfft_plan_create(&p, 2, N, M, n, 6, NFFT_FP64);
    if (rc) {
        printf("nfft_plan_create: %s\n", nfft_strerror(rc));
        return 2;
    }
    if ((rc = nfft_set_nodes_host(p, x)) || (rc = nfft_trafo_host(p, fhat, f)) ||
        (rc = nfft_adjoint_host(p, fv, hh))) {
        printf("transform: %s\n", nfft_strerror(rc));
        nfft_destroy(p);
        return 3;
    }
    double ef = 0, nf = 0, eh = 0, nh = 0;
    for (int j = 0; j < M; j++) { /* direct NDFT, k centred: k_t = idx_t - N_t / 2 */
        double re = 0, im = 0;
        for (int a = 0; a < N0; a++)
            for (int b = 0; b < N1; b++) {
                const double ph = -2 * pi * ((a - N0 / 2) * x[2 * j] + (b - N1 / 2) * x[2 * j + 1]);
                const double cr = fhat[2 * (a * N1 + b)], ci = fhat[2 * (a * N1 + b) + 1];
                re += cr * cos(ph) - ci * sin(ph);
                im += cr * sin(ph) + ci * cos(ph);
            }
        ef += (f[2 * j] - re) * (f[2 * j] - re) + (f[2 * j + 1] - im) * (f[2 * j + 1] - im);
        nf += re * re + im * im;
    }
    for (int a = 0; a < N0; a++)
        for (int b = 0; b < N1; b++) {
            double re = 0, im = 0;
            for (int j = 0; j < M; j++) {
                const double ph = 2 * pi * ((a - N0 / 2) * x[2 * j] + (b - N1 / 2) * x[2 * j + 1]);
                re += fv[2 * j] * cos(ph) - fv[2 * j + 1] * sin(ph);
                im += fv[2 * j] * sin(ph) + fv[2 * j + 1] * cos(ph);
            }
            const int k = a * N1 + b;
            eh += (hh[2 * k] - re) * (hh[2 * k] - re) + (hh[2 * k + 1] - im) * (hh[2 * k + 1] - im);
            nh += re * re + im * im;
        }
    nfft_destroy(p);
    const double rf = sqrt(ef / nf), rh = sqrt(eh / nh);
    printf("%.3e %.3e\n", rf, rh);
    free(x);
    free(fhat);
    free(f);
    free(hh);
    free(fv);
    return (rf < 1e-9 && rh < 1e-9) ? 0 : 1;
}
