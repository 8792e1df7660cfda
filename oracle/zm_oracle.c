/*
 * zm_oracle.c -- plain serial FP64 CPU oracle for the Z-Model interface velocity path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or execute this file;
 * only the test-suite, the smoke check and the benchmark's CPU-baseline leg use it.  It shares
 * no code, header, table or helper with the CUDA library.
 *
 * What it computes (the paper, Beatnik arXiv:2406.05490, names the ingredients but prints no
 * equations; the formulas below are the reading of the Z-Model used throughout this project):
 *
 *   Mesh (Sec. 2 "SurfaceMesh"; Sec. 3.1): n1 x n2 nodes, parameter alpha = (i*dx1, j*dx2),
 *     dx_l = L_l / n_l, node p = i*n2 + j.  Per node: position z = (z1,z2,z3) and two vorticity
 *     components w = (w1,w2).  Arrays are component-major: z[c*N + p], w[c*N + p].
 *   Ghosts (Sec. 3.1 "BoundaryCondition"): two nodes deep.  Periodic: wrap the index and shift
 *     z1 by +-L1 across the alpha1 seam (z2 by +-L2 across the alpha2 seam).  Free edges:
 *     linear extrapolation f(-m) = 2 f(0) - f(m), f(n-1+m) = 2 f(n-1) - f(n-1-m), m = 1, 2.
 *   Stencils (Sec. 3.1 "two-node-deep stencils"): fourth-order central differences
 *     D f = (-f[+2] + 8 f[+1] - 8 f[-1] + f[-2]) / (12 dx)
 *     D2 f = (-f[+2] + 16 f[+1] - 30 f[0] + 16 f[-1] - f[-2]) / (12 dx^2),  Lap = D2_1 + D2_2.
 *   Geometry (Sec. 2 "ZModel": surface normals): a_l = D_l z, h_kl = a_k . a_l,
 *     det = h11 h22 - h12^2, N = a1 x a2 / |a1 x a2|.
 *   Sheet strength: gamma = w1 a2 - w2 a1.
 *   High order (Sec. 2 "BRSolver", Sec. 3.2.1 ExactBRSolver): all-pairs desingularised
 *     Birkhoff-Rott sum
 *       u_i = -(dx1 dx2 / 4 pi) sum_j (z_i - z_j) x gamma_j / (|z_i - z_j|^2 + delta^2)^(3/2).
 *   Low order (Sec. 2: FFT approximation of the Birkhoff-Rott integral): Riesz transforms
 *       s = R1 w1 + R2 w2,  R_l^(k) = -i k_l / |k|,  k_l = 2 pi m_l / L_l,
 *     multiplier zero at k = 0 and on the Nyquist row and column (even sides); u = -1/2 s N.
 *     Sides of any length: radix-2 for powers of two, otherwise Cooley-Tukey on the smallest
 *     prime factor with prime lengths summed by the definition of the DFT.
 *   Cutoff (Sec. 3.2.2 CutoffBRSolver: only the points within a 3D distance of each point):
 *     the same sum restricted to the sources with |z_i - z_j| <= cutoff, decided in FP64 on the
 *     squared distance of the componentwise differences, |z_i - z_j|^2 <= cutoff^2.
 *   Medium order (Sec. 2: couples the FFT and far-field solvers; Sec. 6: uses FFTs for the
 *     change in vorticity): dz/dt = u from the Birkhoff-Rott sum, while Phi (hence dw/dt) takes
 *     the low-order velocity.
 *   Vorticity: Phi = g z3 + 1/8 (h22 w1^2 - 2 h12 w1 w2 + h11 w2^2) / det + 1/2 |u|^2,
 *       dw_l/dt = -2 A D_l Phi + mu Lap w_l,     dz/dt = u.
 *   Time integration (Sec. 3.1 "TimeIntegrator": third-order Runge-Kutta, three derivative
 *     evaluations per step): SSP-RK3 in Shu-Osher form
 *       y1 = y + dt L(y);  y2 = 3/4 y + 1/4 (y1 + dt L(y1));  y' = 1/3 y + 2/3 (y2 + dt L(y2)).
 *
 * All arithmetic is IEEE FP64, compiled without FMA contraction; sums over sources use
 * Neumaier-compensated accumulation.  The default build is serial; an OpenMP build of this same
 * file (liboracle_omp.so) splits only the targets of the Birkhoff-Rott sums across threads and
 * returns the same bits.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "zm_oracle.h"

#define ZMO_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------------ */
/* Ghost-aware node access (Sec. 3.1, BoundaryCondition).                                      */
/* ------------------------------------------------------------------------------------------ */

/* Value of the scalar field f (length n1*n2) at (i, j); at most one of i, j lies in the
 * two-deep halo.  `shift1` / `shift2` is the amount the field jumps by across one period of
 * alpha1 / alpha2 (L1 for z1 along alpha1, L2 for z2 along alpha2, else 0). */
static double node(const zmo_mesh *m, const double *f, int i, int j, double shift1, double shift2)
{
    int n1 = m->n1, n2 = m->n2;
    if (m->periodic) {
        double s = 0.0;
        if (i < 0) { i += n1; s -= shift1; }
        else if (i >= n1) { i -= n1; s += shift1; }
        if (j < 0) { j += n2; s -= shift2; }
        else if (j >= n2) { j -= n2; s += shift2; }
        return f[(size_t)i * n2 + j] + s;
    }
    if (i < 0) return 2.0 * f[(size_t)0 * n2 + j] - f[(size_t)(-i) * n2 + j];
    if (i >= n1) return 2.0 * f[(size_t)(n1 - 1) * n2 + j] - f[(size_t)(2 * (n1 - 1) - i) * n2 + j];
    if (j < 0) return 2.0 * f[(size_t)i * n2 + 0] - f[(size_t)i * n2 + (-j)];
    if (j >= n2) return 2.0 * f[(size_t)i * n2 + (n2 - 1)] - f[(size_t)i * n2 + (2 * (n2 - 1) - j)];
    return f[(size_t)i * n2 + j];
}

/* First derivative along axis (0: alpha1, 1: alpha2), fourth-order central. */
static double d1(const zmo_mesh *m, const double *f, int i, int j, int axis, double shift)
{
    double fp2, fp1, fm1, fm2, dx;
    if (axis == 0) {
        fp2 = node(m, f, i + 2, j, shift, 0.0);
        fp1 = node(m, f, i + 1, j, shift, 0.0);
        fm1 = node(m, f, i - 1, j, shift, 0.0);
        fm2 = node(m, f, i - 2, j, shift, 0.0);
        dx = m->L1 / m->n1;
    } else {
        fp2 = node(m, f, i, j + 2, 0.0, shift);
        fp1 = node(m, f, i, j + 1, 0.0, shift);
        fm1 = node(m, f, i, j - 1, 0.0, shift);
        fm2 = node(m, f, i, j - 2, 0.0, shift);
        dx = m->L2 / m->n2;
    }
    return (-fp2 + 8.0 * fp1 - 8.0 * fm1 + fm2) / (12.0 * dx);
}

/* Second derivative along one axis, fourth-order central (fields without a seam shift). */
static double d2(const zmo_mesh *m, const double *f, int i, int j, int axis)
{
    double fp2, fp1, f0, fm1, fm2, dx;
    f0 = f[(size_t)i * m->n2 + j];
    if (axis == 0) {
        fp2 = node(m, f, i + 2, j, 0.0, 0.0);
        fp1 = node(m, f, i + 1, j, 0.0, 0.0);
        fm1 = node(m, f, i - 1, j, 0.0, 0.0);
        fm2 = node(m, f, i - 2, j, 0.0, 0.0);
        dx = m->L1 / m->n1;
    } else {
        fp2 = node(m, f, i, j + 2, 0.0, 0.0);
        fp1 = node(m, f, i, j + 1, 0.0, 0.0);
        fm1 = node(m, f, i, j - 1, 0.0, 0.0);
        fm2 = node(m, f, i, j - 2, 0.0, 0.0);
        dx = m->L2 / m->n2;
    }
    return (-fp2 + 16.0 * fp1 - 30.0 * f0 + 16.0 * fm1 - fm2) / (12.0 * dx * dx);
}

void zmo_diff1(const zmo_mesh *m, const double *f, double shift, int axis, double *out)
{
    for (int i = 0; i < m->n1; i++)
        for (int j = 0; j < m->n2; j++)
            out[(size_t)i * m->n2 + j] = d1(m, f, i, j, axis, shift);
}

void zmo_laplacian(const zmo_mesh *m, const double *f, double *out)
{
    for (int i = 0; i < m->n1; i++)
        for (int j = 0; j < m->n2; j++)
            out[(size_t)i * m->n2 + j] = d2(m, f, i, j, 0) + d2(m, f, i, j, 1);
}

/* ------------------------------------------------------------------------------------------ */
/* Geometry: tangents, metric, unit normal, sheet strength (Sec. 2, ZModel: surface normals).   */
/* ------------------------------------------------------------------------------------------ */

void zmo_geometry(const zmo_mesh *m, const double *z, double *a1, double *a2, double *h,
                  double *nrm)
{
    size_t N = (size_t)m->n1 * m->n2;
    for (int c = 0; c < 3; c++) {
        double s1 = (c == 0) ? m->L1 : 0.0; /* z1 jumps by L1 across the alpha1 seam */
        double s2 = (c == 1) ? m->L2 : 0.0; /* z2 jumps by L2 across the alpha2 seam */
        zmo_diff1(m, z + c * N, s1, 0, a1 + c * N);
        zmo_diff1(m, z + c * N, s2, 1, a2 + c * N);
    }
    for (size_t p = 0; p < N; p++) {
        double x1 = a1[p], y1 = a1[N + p], w1 = a1[2 * N + p];
        double x2 = a2[p], y2 = a2[N + p], w2 = a2[2 * N + p];
        double h11 = x1 * x1 + y1 * y1 + w1 * w1;
        double h12 = x1 * x2 + y1 * y2 + w1 * w2;
        double h22 = x2 * x2 + y2 * y2 + w2 * w2;
        if (h) {
            h[p] = h11;
            h[N + p] = h12;
            h[2 * N + p] = h22;
            h[3 * N + p] = h11 * h22 - h12 * h12;
        }
        if (nrm) {
            double cx = y1 * w2 - w1 * y2;
            double cy = w1 * x2 - x1 * w2;
            double cz = x1 * y2 - y1 * x2;
            double len = sqrt(cx * cx + cy * cy + cz * cz);
            nrm[p] = cx / len;
            nrm[N + p] = cy / len;
            nrm[2 * N + p] = cz / len;
        }
    }
}

void zmo_sheet_strength(size_t N, const double *w, const double *a1, const double *a2,
                        double *gamma)
{
    for (size_t p = 0; p < N; p++)
        for (int c = 0; c < 3; c++)
            gamma[c * N + p] = w[p] * a2[c * N + p] - w[N + p] * a1[c * N + p];
}

/* ------------------------------------------------------------------------------------------ */
/* High order: exact all-pairs Birkhoff-Rott sum (Sec. 3.2.1, ExactBRSolver).                   */
/* ------------------------------------------------------------------------------------------ */

/* Neumaier (improved Kahan) compensated accumulation. */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

void zmo_br_velocity(size_t nt, const double *zt, size_t ns, const double *zs,
                     const double *gamma, double weight, double delta, double *u)
{
    double pref = -weight / (4.0 * ZMO_PI);
    double d2 = delta * delta;
    /* Targets are independent and each one's sum runs in the same order either way, so an
     * OpenMP build (used only to write stored expected states faster) gives identical bits. */
#pragma omp parallel for schedule(dynamic, 64)
    for (size_t i = 0; i < nt; i++) {
        nsum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
        double xi = zt[i], yi = zt[nt + i], wi = zt[2 * nt + i];
        for (size_t j = 0; j < ns; j++) {
            double rx = xi - zs[j], ry = yi - zs[ns + j], rz = wi - zs[2 * ns + j];
            double gx = gamma[j], gy = gamma[ns + j], gz = gamma[2 * ns + j];
            double r2 = rx * rx + ry * ry + rz * rz + d2;
            double k = 1.0 / (r2 * sqrt(r2)); /* (|r|^2 + delta^2)^(-3/2) */
            /* (z_i - z_j) x gamma_j */
            nadd(&acc[0], (ry * gz - rz * gy) * k);
            nadd(&acc[1], (rz * gx - rx * gz) * k);
            nadd(&acc[2], (rx * gy - ry * gx) * k);
        }
        for (int c = 0; c < 3; c++) u[c * nt + i] = pref * (acc[c].s + acc[c].c);
    }
}

/* Cutoff decision (Sec. 3.2.2): source z_j (component stride sj) counts for target z_i
 * (stride si) iff its distance is at most the cutoff, |z_i - z_j|^2 <= cutoff^2 in FP64. */
int zmo_within_cutoff(const double *zi, size_t si, const double *zj, size_t sj, double cutoff)
{
    double dist2 = 0.0;
    for (int c = 0; c < 3; c++) {
        double d = zi[c * si] - zj[c * sj];
        dist2 += d * d;
    }
    return dist2 <= cutoff * cutoff;
}

void zmo_br_velocity_cutoff(size_t nt, const double *zt, size_t ns, const double *zs,
                            const double *gamma, double weight, double delta, double cutoff,
                            double *u)
{
    double pref = -weight / (4.0 * ZMO_PI);
    double d2 = delta * delta;
#pragma omp parallel for schedule(dynamic, 64)
    for (size_t i = 0; i < nt; i++) {
        nsum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
        double xi = zt[i], yi = zt[nt + i], wi = zt[2 * nt + i];
        for (size_t j = 0; j < ns; j++) {
            if (!zmo_within_cutoff(zt + i, nt, zs + j, ns, cutoff)) continue;
            double rx = xi - zs[j], ry = yi - zs[ns + j], rz = wi - zs[2 * ns + j];
            double gx = gamma[j], gy = gamma[ns + j], gz = gamma[2 * ns + j];
            double r2 = rx * rx + ry * ry + rz * rz + d2;
            double k = 1.0 / (r2 * sqrt(r2));
            nadd(&acc[0], (ry * gz - rz * gy) * k);
            nadd(&acc[1], (rz * gx - rx * gz) * k);
            nadd(&acc[2], (rx * gy - ry * gx) * k);
        }
        for (int c = 0; c < 3; c++) u[c * nt + i] = pref * (acc[c].s + acc[c].c);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Low order: FFT Riesz-transform velocity (Sec. 2: FFT approximation of the BR integral).      */
/* ------------------------------------------------------------------------------------------ */

/* In-place iterative radix-2 FFT of one complex sequence of power-of-two length n, accessed
 * with a stride.  sign = -1: forward X_k = sum_m x_m exp(-2 pi i k m / n); sign = +1: the
 * unnormalised inverse. */
static void fft1d(int n, double *re, double *im, size_t stride, int sign)
{
    for (int a = 1, b = 0; a < n; a++) { /* bit-reversal permutation */
        int bit = n >> 1;
        for (; b & bit; bit >>= 1) b ^= bit;
        b ^= bit;
        if (a < b) {
            double t = re[a * stride]; re[a * stride] = re[b * stride]; re[b * stride] = t;
            t = im[a * stride]; im[a * stride] = im[b * stride]; im[b * stride] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        for (int k = 0; k < len / 2; k++) {
            double ang = sign * 2.0 * ZMO_PI * k / len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < n; s += len) {
                size_t p = (size_t)(s + k) * stride, q = (size_t)(s + k + len / 2) * stride;
                double xr = re[q] * wr - im[q] * wi;
                double xi = re[q] * wi + im[q] * wr;
                re[q] = re[p] - xr; im[q] = im[p] - xi;
                re[p] += xr; im[p] += xi;
            }
        }
    }
}

/* Any length n (Cooley-Tukey, decimation in time, split on the smallest prime factor p of n;
 * a prime length is summed by the definition).  With n = p m and x_q[t] = x[t p + q]:
 *     X[k] = sum_q W_n^(q k) Y_q[k mod m],   Y_q = DFT_m(x_q),   W_n = exp(sign 2 pi i / n).
 * `wr`, `wi` hold W_ntop^t for t < ntop, with n dividing ntop: W_n^e = W_ntop^(e ntop / n).
 * Input x (stride `stride`), output X (contiguous), scratch of 2n doubles per level. */
static void dft_any(int n, const double *xr, const double *xi, size_t stride, double *yr,
                    double *yi, int ntop, const double *wr, const double *wi)
{
    int p = 2;
    while (p * p <= n && n % p) p++;
    if (n % p) p = n; /* n is prime (or 1) */
    const int m = n / p, scale = ntop / n;
    if (p == n) {
        for (int k = 0; k < n; k++) {
            double sr = 0.0, si = 0.0;
            for (int t = 0; t < n; t++) {
                const size_t e = (size_t)((long long)t * k % n) * scale;
                const double ar = xr[t * stride], ai = xi[t * stride];
                sr += ar * wr[e] - ai * wi[e];
                si += ar * wi[e] + ai * wr[e];
            }
            yr[k] = sr;
            yi[k] = si;
        }
        return;
    }
    double *sub = malloc(2 * (size_t)n * sizeof(double)); /* Y_q for q < p, each of length m */
    for (int q = 0; q < p; q++)
        dft_any(m, xr + q * stride, xi + q * stride, stride * p, sub + (size_t)q * m,
                sub + (size_t)n + (size_t)q * m, ntop, wr, wi);
    for (int k = 0; k < n; k++) {
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < p; q++) {
            const size_t e = (size_t)((long long)q * k % n) * scale;
            const double ar = sub[(size_t)q * m + k % m], ai = sub[(size_t)n + (size_t)q * m + k % m];
            sr += ar * wr[e] - ai * wi[e];
            si += ar * wi[e] + ai * wr[e];
        }
        yr[k] = sr;
        yi[k] = si;
    }
    free(sub);
}

/* One complex sequence of any length n >= 1 in place (stride `stride`), sign as in fft1d:
 * powers of two go through fft1d, other lengths through dft_any. */
static void fft1d_any(int n, double *re, double *im, size_t stride, int sign, const double *wr,
                      const double *wi)
{
    if ((n & (n - 1)) == 0) {
        fft1d(n, re, im, stride, sign);
        return;
    }
    double *yr = malloc(2 * (size_t)n * sizeof(double)), *yi = yr + n;
    dft_any(n, re, im, stride, yr, yi, n, wr, wi);
    for (int k = 0; k < n; k++) {
        re[k * stride] = yr[k];
        im[k * stride] = yi[k];
    }
    free(yr);
}

/* W_n^t = exp(sign 2 pi i t / n), t < n, into wr[t], wi[t]. */
static void roots(int n, int sign, double *wr, double *wi)
{
    for (int t = 0; t < n; t++) {
        const double ang = sign * 2.0 * ZMO_PI * t / n;
        wr[t] = cos(ang);
        wi[t] = sin(ang);
    }
}

void zmo_fft2(int n1, int n2, double *re, double *im, int sign)
{
    double *w1 = malloc(2 * (size_t)n1 * sizeof(double)), *w2 = malloc(2 * (size_t)n2 * sizeof(double));
    roots(n1, sign, w1, w1 + n1);
    roots(n2, sign, w2, w2 + n2);
    for (int i = 0; i < n1; i++)
        fft1d_any(n2, re + (size_t)i * n2, im + (size_t)i * n2, 1, sign, w2, w2 + n2);
    for (int j = 0; j < n2; j++) fft1d_any(n1, re + j, im + j, (size_t)n2, sign, w1, w1 + n1);
    free(w1);
    free(w2);
}

/* Signed frequency of DFT index idx: 0, 1, .., then negative from the middle on (for even n the
 * middle index n/2 maps to -n/2, the Nyquist frequency, whose multiplier is zero). */
static int signed_freq(int idx, int n) { return 2 * idx < n ? idx : idx - n; }

void zmo_riesz_scalar(const zmo_mesh *m, const double *w, double *s)
{
    int n1 = m->n1, n2 = m->n2;
    size_t N = (size_t)n1 * n2;
    double *r1 = calloc(N, sizeof(double)), *i1 = calloc(N, sizeof(double));
    double *r2 = calloc(N, sizeof(double)), *i2 = calloc(N, sizeof(double));
    memcpy(r1, w, N * sizeof(double));
    memcpy(r2, w + N, N * sizeof(double));
    zmo_fft2(n1, n2, r1, i1, -1);
    zmo_fft2(n1, n2, r2, i2, -1);
    for (int a = 0; a < n1; a++) {
        for (int b = 0; b < n2; b++) {
            size_t p = (size_t)a * n2 + b;
            int m1 = signed_freq(a, n1), m2 = signed_freq(b, n2);
            double sr = 0.0, si = 0.0;
            if (!(m1 == 0 && m2 == 0) && 2 * a != n1 && 2 * b != n2) {
                double k1 = 2.0 * ZMO_PI * m1 / m->L1, k2 = 2.0 * ZMO_PI * m2 / m->L2;
                double kk = sqrt(k1 * k1 + k2 * k2);
                /* s^ = R1^ w1^ + R2^ w2^ with R_l^ = -i k_l/|k|:  -i c (x + i y) = c (y - i x) */
                double c1 = k1 / kk, c2 = k2 / kk;
                sr = c1 * i1[p] + c2 * i2[p];
                si = -(c1 * r1[p] + c2 * r2[p]);
            }
            r1[p] = sr;
            i1[p] = si;
        }
    }
    zmo_fft2(n1, n2, r1, i1, +1);
    for (size_t p = 0; p < N; p++) s[p] = r1[p] / (double)N;
    free(r1); free(i1); free(r2); free(i2);
}

/* ------------------------------------------------------------------------------------------ */
/* Vorticity derivative and the full derivative L(z, w).                                        */
/* ------------------------------------------------------------------------------------------ */

void zmo_phi(size_t N, const double *z, const double *w, const double *h, const double *u,
             double g, double *phi)
{
    for (size_t p = 0; p < N; p++) {
        double w1 = w[p], w2 = w[N + p];
        double h11 = h[p], h12 = h[N + p], h22 = h[2 * N + p], det = h[3 * N + p];
        double jump = (h22 * w1 * w1 - 2.0 * h12 * w1 * w2 + h11 * w2 * w2) / det;
        double uu = u[p] * u[p] + u[N + p] * u[N + p] + u[2 * N + p] * u[2 * N + p];
        phi[p] = g * z[2 * N + p] + 0.125 * jump + 0.5 * uu;
    }
}

void zmo_wdot(const zmo_mesh *m, const double *phi, const double *w, double atwood, double mu,
              double *wdot)
{
    size_t N = (size_t)m->n1 * m->n2;
    double *tmp = malloc(N * sizeof(double));
    for (int l = 0; l < 2; l++) {
        zmo_diff1(m, phi, 0.0, l, wdot + l * N);
        for (size_t p = 0; p < N; p++) wdot[l * N + p] *= -2.0 * atwood;
        if (mu != 0.0) {
            zmo_laplacian(m, w + l * N, tmp);
            for (size_t p = 0; p < N; p++) wdot[l * N + p] += mu * tmp[p];
        }
    }
    free(tmp);
}

int zmo_derivative(const zmo_mesh *m, const zmo_params *prm, const double *z, const double *w,
                   double *u, double *wdot)
{
    size_t N = (size_t)m->n1 * m->n2;
    double *a1 = malloc(3 * N * sizeof(double)), *a2 = malloc(3 * N * sizeof(double));
    double *h = malloc(4 * N * sizeof(double)), *nrm = malloc(3 * N * sizeof(double));
    double *phi = malloc(N * sizeof(double));
    zmo_geometry(m, z, a1, a2, h, nrm);
    double *u_low = NULL;  /* the velocity Phi uses */
    if (prm->order != ZMO_ORDER_HIGH) {
        double *s = malloc(N * sizeof(double));
        u_low = malloc(3 * N * sizeof(double));
        zmo_riesz_scalar(m, w, s);
        for (size_t p = 0; p < N; p++)
            for (int c = 0; c < 3; c++) u_low[c * N + p] = -0.5 * s[p] * nrm[c * N + p];
        free(s);
    }
    if (prm->order != ZMO_ORDER_LOW) {
        double *gamma = malloc(3 * N * sizeof(double));
        zmo_sheet_strength(N, w, a1, a2, gamma);
        double weight = (m->L1 / m->n1) * (m->L2 / m->n2);
        if (prm->cutoff > 0)
            zmo_br_velocity_cutoff(N, z, N, z, gamma, weight, prm->delta, prm->cutoff, u);
        else
            zmo_br_velocity(N, z, N, z, gamma, weight, prm->delta, u);
        free(gamma);
    } else {
        memcpy(u, u_low, 3 * N * sizeof(double));
    }
    zmo_phi(N, z, w, h, u_low ? u_low : u, prm->g, phi);
    free(u_low);
    if (wdot) zmo_wdot(m, phi, w, prm->atwood, prm->mu, wdot);
    free(a1); free(a2); free(h); free(nrm); free(phi);
    return 0;
}

/* One SSP-RK3 (Shu-Osher) step of (z, w) in place (Sec. 3.1, TimeIntegrator). */
int zmo_rk3_step(const zmo_mesh *m, const zmo_params *prm, double *z, double *w, double dt)
{
    size_t N = (size_t)m->n1 * m->n2;
    size_t S = 5 * N; /* state vector y = (z1, z2, z3, w1, w2) */
    double *y0 = malloc(S * sizeof(double)), *y = malloc(S * sizeof(double));
    double *ydot = malloc(S * sizeof(double));
    static const double a[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double b[3] = {1.0, 0.25, 2.0 / 3.0};
    memcpy(y0, z, 3 * N * sizeof(double));
    memcpy(y0 + 3 * N, w, 2 * N * sizeof(double));
    memcpy(y, y0, S * sizeof(double));
    for (int stage = 0; stage < 3; stage++) {
        /* L(y): dz/dt = u, dw/dt = wdot */
        zmo_derivative(m, prm, y, y + 3 * N, ydot, ydot + 3 * N);
        for (size_t k = 0; k < S; k++)
            y[k] = a[stage] * y0[k] + b[stage] * (y[k] + dt * ydot[k]);
    }
    memcpy(z, y, 3 * N * sizeof(double));
    memcpy(w, y + 3 * N, 2 * N * sizeof(double));
    free(y0); free(y); free(ydot);
    return 0;
}

int zmo_run(const zmo_mesh *m, const zmo_params *prm, double *z, double *w, double dt,
            int nsteps)
{
    for (int s = 0; s < nsteps; s++) zmo_rk3_step(m, prm, z, w, dt);
    return 0;
}
