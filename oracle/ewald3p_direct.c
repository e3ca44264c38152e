/*
 * FP64 direct evaluation of the triply periodic Ewald sums (Ewald3P).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a reference ("oracle") the CUDA path
 * is checked against; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may build, load or call it.  It shares no code,
 * header or constant with the GPU library.
 *
 * The SE1P paper measures its method against the triply periodic Spectral
 * Ewald method (SE3P, Section 1 and Example 6.5), which approximates the
 * classical Ewald3P sums for a neutral system in a box periodic in x, y and z
 * (tin-foil boundary, no k = 0 term):
 *
 *   phi(x_m) = phi^R + phi^F + phi^self
 *   phi^R    = sum'_{p in Z^3} sum_n q_n erfc(xi r)/r,  r = |x_m - x_n + p L|, r <= rc
 *   phi^F    = (4 pi / V) sum_{k != 0} e^{-k^2/4xi^2} / k^2  sum_n q_n cos(k . (x_m - x_n)),
 *              k = 2 pi (j1/L1, j2/L2, j3/L3), truncated where e^{-k^2/4xi^2} < kcut
 *   phi^self = -2 xi / sqrt(pi) q_m
 *
 * Forces F_m = -q_m grad_m phi(x_m), the gradient acting on the target only:
 *   F^R = q_m sum q_n (erfc(xi r)/r + 2 xi/sqrt(pi) e^{-xi^2 r^2}) r_vec / r^2
 *   F^F = q_m (4 pi / V) sum_k e^{-k^2/4xi^2}/k^2  k  sum_n q_n sin(k . (x_m - x_n))
 *
 * The k-space sum uses the structure factor S(k) = sum_n q_n e^{-i k . x_n}, so
 * that sum_n q_n e^{i k . (x_m - x_n)} = e^{i k . x_m} S(k); k and -k are taken
 * together (half of the lattice, doubled).
 */
#include <math.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define E3_PI 3.14159265358979323846264338327950288

/* Returns 0 on success, -1 on invalid arguments, -2 if memory ran out.
 * phi: [nt][3] (R, F, self); frc: [nt][2][3] (R, F). */
int orc_ewald3p(int n, const double *x, const double *q, int nt, const int *tgt, const double *L, double xi,
                double rc, double kcut, double *phi, double *frc)
{
    if (n < 0 || nt < 0 || !(xi > 0.0) || !(kcut > 0.0) || kcut >= 1.0) return -1;
    for (int d = 0; d < 3; ++d)
        if (!(L[d] > 0.0)) return -1;
    const double V = L[0] * L[1] * L[2];
    const double sqpi = sqrt(E3_PI);

    /* ---- k-space: lattice vectors of the half space (j3 > 0, or j3 = 0 and j2 > 0, or j3 = j2 = 0, j1 > 0) */
    const double kmax2 = -4.0 * xi * xi * log(kcut);
    int jm[3];
    for (int d = 0; d < 3; ++d) jm[d] = (int)ceil(sqrt(kmax2) * L[d] / (2.0 * E3_PI));
    long nk_max = (long)(2 * jm[0] + 1) * (2 * jm[1] + 1) * (jm[2] + 1);
    double *kv = (double *)malloc(sizeof(double) * 4 * (size_t)nk_max); /* kx, ky, kz, weight */
    double *sre = (double *)malloc(sizeof(double) * (size_t)nk_max);
    double *sim = (double *)malloc(sizeof(double) * (size_t)nk_max);
    if (!kv || !sre || !sim) {
        free(kv);
        free(sre);
        free(sim);
        return -2;
    }
    long nk = 0;
    for (int j3 = 0; j3 <= jm[2]; ++j3)
        for (int j2 = -jm[1]; j2 <= jm[1]; ++j2)
            for (int j1 = -jm[0]; j1 <= jm[0]; ++j1) {
                if (j3 == 0 && (j2 < 0 || (j2 == 0 && j1 <= 0))) continue;
                const double kx = 2.0 * E3_PI * j1 / L[0], ky = 2.0 * E3_PI * j2 / L[1], kz = 2.0 * E3_PI * j3 / L[2];
                const double k2 = kx * kx + ky * ky + kz * kz;
                if (k2 > kmax2) continue;
                kv[4 * nk] = kx;
                kv[4 * nk + 1] = ky;
                kv[4 * nk + 2] = kz;
                kv[4 * nk + 3] = 2.0 * (4.0 * E3_PI / V) * exp(-k2 / (4.0 * xi * xi)) / k2; /* k and -k */
                ++nk;
            }
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < nk; ++k) {
        double a = 0.0, b = 0.0;
        for (int s = 0; s < n; ++s) {
            const double ph = kv[4 * k] * x[3 * s] + kv[4 * k + 1] * x[3 * s + 1] + kv[4 * k + 2] * x[3 * s + 2];
            a += q[s] * cos(ph);
            b -= q[s] * sin(ph);
        }
        sre[k] = a;
        sim[k] = b;
    }

    /* ---- per target */
    int im[3];
    for (int d = 0; d < 3; ++d) im[d] = rc > 0.0 ? (int)ceil(rc / L[d]) + 1 : 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < nt; ++t) {
        const int m = tgt ? tgt[t] : t;
        const double xm = x[3 * m], ym = x[3 * m + 1], zm = x[3 * m + 2];
        double pr = 0.0, fr[3] = {0.0, 0.0, 0.0};
        if (rc > 0.0) {
            for (int s = 0; s < n; ++s) {
                for (int a = -im[0]; a <= im[0]; ++a)
                    for (int b = -im[1]; b <= im[1]; ++b)
                        for (int c = -im[2]; c <= im[2]; ++c) {
                            const double dx = xm - x[3 * s] + a * L[0];
                            const double dy = ym - x[3 * s + 1] + b * L[1];
                            const double dz = zm - x[3 * s + 2] + c * L[2];
                            const double r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 == 0.0 || r2 > rc * rc) continue;
                            const double r = sqrt(r2);
                            const double e = erfc(xi * r) / r;
                            pr += q[s] * e;
                            const double fs = q[s] * (e + 2.0 * xi / sqpi * exp(-xi * xi * r2)) / r2;
                            fr[0] += fs * dx;
                            fr[1] += fs * dy;
                            fr[2] += fs * dz;
                        }
            }
        }
        double pf = 0.0, ff[3] = {0.0, 0.0, 0.0};
        for (long k = 0; k < nk; ++k) {
            const double ph = kv[4 * k] * xm + kv[4 * k + 1] * ym + kv[4 * k + 2] * zm;
            const double c = cos(ph), sn = sin(ph);
            /* e^{i k x_m} S(k) = (c + i sn)(sre + i sim) */
            const double re = c * sre[k] - sn * sim[k];
            const double imv = c * sim[k] + sn * sre[k];
            pf += kv[4 * k + 3] * re;
            for (int d = 0; d < 3; ++d) ff[d] += kv[4 * k + 3] * kv[4 * k + d] * imv;
        }
        phi[3 * t] = pr;
        phi[3 * t + 1] = pf;
        phi[3 * t + 2] = -2.0 * xi / sqpi * q[m];
        for (int d = 0; d < 3; ++d) {
            frc[6 * t + d] = q[m] * fr[d];
            frc[6 * t + 3 + d] = q[m] * ff[d];
        }
    }
    free(kv);
    free(sre);
    free(sim);
    return 0;
}
