/*
 * FP64 direct evaluation of the singly periodic Ewald sums (Ewald1P).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference ("oracle") the CUDA
 * path is checked against.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may build, load or call it.  It shares no code,
 * header or constant with the GPU library.
 *
 * What it computes (Section 2.1 of Saffar Shamshirgar & Tornberg, "The
 * Spectral Ewald method for singly periodic domains"), for a box periodic in z
 * with period L3 and free in x,y:
 *
 *   phi(x_m) = phi^R + phi^{F,k3!=0} + phi^{F,k3=0} + phi^self           (Eq. 2.1)
 *   phi^R        = sum'_{alpha} sum_n q_n erfc(xi r)/r, r=|x_m-x_n+alpha L3 e_z|,
 *                  truncated at r <= rc                                   (Eq. 2.2)
 *   phi^{k3!=0}  = (1/L3) sum_{k3!=0} sum_n q_n e^{i k3 dz} K0(k3^2/4xi^2, xi^2 rho^2)
 *                = (2/L3) sum_{j>=1} sum_n q_n cos(k_j dz) K0(a_j, b)       (Eq. 2.3b)
 *   phi^{k3=0}   = -(1/L3) sum_{n!=m} q_n [gamma + log(xi^2 rho^2) + E1(xi^2 rho^2)]  (Eq. 2.4)
 *   phi^self     = -2 xi/sqrt(pi) q_m                                     (Eq. 2.5)
 *
 * Forces are F_m = -q_m grad_m phi(x_m), the gradient acting on the target
 * position only.  This is the reading under which the force is minus the
 * gradient of U = 1/2 sum_m q_m phi_m (Section 3.5 prints both a factor 1/2
 * and 1/L3 in the k3=0 force, Eq. 3.24; differentiating Eq. 2.4 gives 2/L3).
 *
 * Special functions (Appendix A):
 *   E1(x):   power series for x < 1 (Eq. A.4), continued fraction for
 *            x >= 1 (Eq. A.2 with n = 1), evaluated by the modified Lentz
 *            recurrence.
 *   K0(a,b): the incomplete Bessel function int_1^inf t^-1 e^{-a t - b/t} dt.
 *            With t = e^u it is int_0^inf exp(-a e^u - b e^-u) du, an
 *            integrand with a single maximum at u* = max(0, log(b/a)/2); the
 *            oracle integrates it with composite 20-point Gauss-Legendre
 *            panels placed around u* (width tied to the local curvature),
 *            until the integrand has fallen by e^-60.  The paper splits the
 *            t-interval instead; both are quadratures of the same definition.
 *   dK0/db = -int_1^inf t^-2 e^{-a t - b/t} dt = -int_0^inf e^-u exp(...) du.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288
#define ORC_EULER_GAMMA 0.57721566490153286060651209008240243

/* ---------------------------------------------------------------- Gauss-Legendre nodes */
#define GL_N 20
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

/* Nodes/weights of the 20-point Gauss-Legendre rule on [-1,1]: Newton's method
 * on P_20 from the Chebyshev-like initial guess, with P_n and P_n' from the
 * three-term recurrence. */
static void gl_init(void)
{
    if (gl_ready) return;
    for (int i = 0; i < GL_N; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (GL_N + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= GL_N; ++k) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = GL_N * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        gl_x[i] = z;
        gl_w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    gl_ready = 1;
}

/* ---------------------------------------------------------------- E1 and g */

/* E1(x) for x > 0 (Appendix A, Eqs. A.2 and A.4). */
double orc_e1(double x)
{
    if (!(x > 0.0)) return INFINITY;
    if (x < 1.0) {
        /* E1 = -gamma - log x - sum_{m>=1} (-x)^m / (m m!) */
        double term = 1.0, sum = 0.0;
        for (int m = 1; m < 200; ++m) {
            term *= -x / m; /* (-x)^m / m! */
            double t = term / m;
            sum += t;
            if (fabs(t) < 1e-18 * fabs(sum)) break;
        }
        return -ORC_EULER_GAMMA - log(x) - sum;
    }
    /* E1 = e^-x * 1/(x+1- 1^2/(x+3- 2^2/(x+5- ...))) by modified Lentz. */
    const double tiny = 1e-300;
    double b = x + 1.0;
    double c = 1.0 / tiny;
    double d = 1.0 / b;
    double h = d;
    for (int i = 1; i < 10000; ++i) {
        double an = -(double)i * (double)i;
        b += 2.0;
        d = 1.0 / (an * d + b);
        c = b + an / c;
        double del = c * d;
        h *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    return h * exp(-x);
}

/* g(u) = gamma + log u + E1(u), the k3=0 kernel of Eq. 2.4; g(0) = 0 (Eq. A.5).
 * For u < 1 the series -sum_{m>=1} (-u)^m/(m m!) avoids the cancellation. */
double orc_g(double u)
{
    if (u <= 0.0) return 0.0;
    if (u < 1.0) {
        double term = 1.0, sum = 0.0;
        for (int m = 1; m < 200; ++m) {
            term *= -u / m;
            double t = term / m;
            sum += t;
            if (fabs(t) < 1e-18 * fabs(sum)) break;
        }
        return -sum;
    }
    return ORC_EULER_GAMMA + log(u) + orc_e1(u);
}

/* ---------------------------------------------------------------- incomplete Bessel K0(a,b) */

/* int_0^inf e^{-p u} exp(-a e^u - b e^-u) du for p = 0 (K0) or p = 1 (-dK0/db). a > 0, b >= 0. */
static double kinc_quad(double a, double b, int p)
{
    gl_init();
    double u0 = 0.0;
    if (b > a) u0 = 0.5 * log(b / a);
    const double phi0 = a * exp(u0) + b * exp(-u0); /* also phi''(u0) */
    const double drop = 60.0;
    /* width of the peak; panels span at most 2 widths (and at most 1) */
    double w = 2.0 / sqrt(phi0 > 1e-300 ? phi0 : 1e-300);
    if (w > 1.0) w = 1.0;
    /* right end: phi(u) - phi0 > drop */
    double hi = u0;
    while (a * exp(hi) + b * exp(-hi) - phi0 < drop) hi += w;
    /* left end: stop at 0 or where phi has risen by drop */
    double lo = u0;
    while (lo > 0.0 && a * exp(lo) + b * exp(-lo) - phi0 < drop) lo -= w;
    if (lo < 0.0) lo = 0.0;
    int npan = (int)ceil((hi - lo) / w);
    if (npan < 1) npan = 1;
    double pw = (hi - lo) / npan;
    double sum = 0.0;
    for (int k = 0; k < npan; ++k) {
        double c = lo + (k + 0.5) * pw;
        double s = 0.0;
        for (int i = 0; i < GL_N; ++i) {
            double u = c + 0.5 * pw * gl_x[i];
            double eu = exp(u);
            double f = exp(-a * eu - b / eu);
            if (p) f /= eu;
            s += gl_w[i] * f;
        }
        sum += 0.5 * pw * s;
    }
    return sum;
}

double orc_kinc(double a, double b) { return kinc_quad(a, b, 0); }

/* -dK0(a,b)/db */
double orc_kinc_mdb(double a, double b) { return kinc_quad(a, b, 1); }

/* ---------------------------------------------------------------- Ewald1P direct sums */

/*
 * Evaluate the four potential parts and three force parts at the targets.
 *
 *   n, x[3n], q[n]   sources (x,y free, z periodic with period L3)
 *   nt, tgt[nt]      target indices into the sources (tgt == NULL: all n)
 *   L3, xi, rc       period, Ewald parameter, real-space cutoff (rc <= 0: skip phi^R)
 *   kcut             k3 != 0 modes with e^{-a}/a < kcut are dropped (a = k3^2/4xi^2)
 *   phi_out[4 nt]    per target: phi^R, phi^{F,k3!=0}, phi^{F,k3=0}, phi^self
 *   frc_out[9 nt]    per target: F^R (3), F^{F,k3!=0} (3), F^{F,k3=0} (3)
 *
 * Returns 0, or -1 on bad arguments.
 */
int orc_ewald1p(int n, const double *x, const double *q, int nt, const int *tgt, double L3,
                double xi, double rc, double kcut, double *phi_out, double *frc_out)
{
    if (n < 0 || nt < 0 || !(L3 > 0.0) || !(xi > 0.0) || !phi_out || !frc_out) return -1;
    gl_init();
    const double xi2 = xi * xi;
    const double two_xi_sqpi = 2.0 * xi / sqrt(ORC_PI);
    /* number of k3 > 0 modes kept */
    int jmax = 0;
    for (int j = 1; j < 1000000; ++j) {
        double k = 2.0 * ORC_PI * j / L3;
        double a = k * k / (4.0 * xi2);
        if (exp(-a) / a < kcut) break;
        jmax = j;
    }
    /* z images that can lie within rc of a principal offset: |alpha L3| <= rc + L3/2 */
    int amax = rc > 0.0 ? (int)ceil(rc / L3) + 1 : 0;

    /* Work items are (target, source chunk) pairs so that a few targets still keep
     * every thread busy; each item writes its partial sums, which are then added
     * in a fixed order (the result does not depend on the thread count). */
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    int nchunk = 1;
    if (nt > 0 && nt < 4 * nthr) nchunk = (4 * nthr + nt - 1) / nt;
    if (nchunk > n) nchunk = n > 0 ? n : 1;
    const int chunk = n > 0 ? (n + nchunk - 1) / nchunk : 0;
    double *part = (double *)calloc((size_t)nt * nchunk * 12, sizeof(double));
    if (!part && nt > 0) return -1;

#pragma omp parallel for schedule(dynamic, 1)
    for (long item = 0; item < (long)nt * nchunk; ++item) {
        const int it = (int)(item / nchunk), ic = (int)(item % nchunk);
        const int m = tgt ? tgt[it] : it;
        const int n0 = ic * chunk, n1 = n0 + chunk < n ? n0 + chunk : n;
        const double xm = x[3 * m], ym = x[3 * m + 1], zm = x[3 * m + 2];
        double pR = 0, pK = 0, p0 = 0;
        double fR[3] = {0, 0, 0}, fK[3] = {0, 0, 0}, f0[3] = {0, 0, 0};
        for (int nn = n0; nn < n1; ++nn) {
            const double qn = q[nn];
            const double dx = xm - x[3 * nn], dy = ym - x[3 * nn + 1], dz = zm - x[3 * nn + 2];
            const double rho2 = dx * dx + dy * dy;
            /* real space, Eq. 2.2 and Eq. 3.22: images of the principal z offset
             * (|dzr| <= L3/2, so any z may be given, not only z in [0, L3)) */
            const double dzr = dz - L3 * rint(dz / L3);
            for (int al = -amax; al <= amax && rc > 0.0; ++al) {
                if (nn == m && al == 0) continue;
                const double dzp = dzr + al * L3;
                const double r2 = rho2 + dzp * dzp;
                const double r = sqrt(r2);
                if (r > rc) continue;
                const double e = erfc(xi * r) / r;
                pR += qn * e;
                const double fs = qn * (two_xi_sqpi * exp(-xi2 * r2) + e) / r2;
                fR[0] += fs * dx;
                fR[1] += fs * dy;
                fR[2] += fs * dzp;
            }
            /* k3 != 0, Eq. 2.3b (n == m included: rho = 0, K0(a,0) = E1(a)) */
            const double b = xi2 * rho2;
            for (int j = 1; j <= jmax; ++j) {
                const double k = 2.0 * ORC_PI * j / L3;
                const double a = k * k / (4.0 * xi2);
                const double K = orc_kinc(a, b);
                const double cs = cos(k * dz), sn = sin(k * dz);
                pK += qn * cs * K;
                /* -grad_m of cos(k dz) K0(a, xi^2 rho^2):
                 *   z:  k sin(k dz) K0 ;  r:  -cos(k dz) 2 xi^2 dr dK0/db */
                fK[2] += qn * k * sn * K;
                if (rho2 > 0.0) {
                    const double D = orc_kinc_mdb(a, b);
                    fK[0] += qn * cs * 2.0 * xi2 * dx * D;
                    fK[1] += qn * cs * 2.0 * xi2 * dy * D;
                }
            }
            /* k3 = 0, Eq. 2.4 */
            if (nn != m) {
                p0 += qn * orc_g(b);
                if (rho2 > 0.0) {
                    const double fz = qn * (-expm1(-b)) / rho2;
                    f0[0] += fz * dx;
                    f0[1] += fz * dy;
                }
            }
        }
        double *o = part + ((size_t)it * nchunk + ic) * 12;
        o[0] = pR;
        o[1] = pK;
        o[2] = p0;
        for (int d = 0; d < 3; ++d) {
            o[3 + d] = fR[d];
            o[6 + d] = fK[d];
            o[9 + d] = f0[d];
        }
    }
    for (int it = 0; it < nt; ++it) {
        const int m = tgt ? tgt[it] : it;
        double acc[12] = {0};
        for (int ic = 0; ic < nchunk; ++ic)
            for (int v = 0; v < 12; ++v) acc[v] += part[((size_t)it * nchunk + ic) * 12 + v];
        const double qm = q[m];
        phi_out[4 * it + 0] = acc[0];
        phi_out[4 * it + 1] = 2.0 / L3 * acc[1];
        phi_out[4 * it + 2] = -1.0 / L3 * acc[2];
        phi_out[4 * it + 3] = -two_xi_sqpi * qm;
        for (int d = 0; d < 3; ++d) {
            frc_out[9 * it + d] = qm * acc[3 + d];
            frc_out[9 * it + 3 + d] = qm * 2.0 / L3 * acc[6 + d];
            frc_out[9 * it + 6 + d] = qm * 2.0 / L3 * acc[9 + d];
        }
    }
    free(part);
    return 0;
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
