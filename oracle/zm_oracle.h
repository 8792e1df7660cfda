/*
 * zm_oracle.h -- declarations of the serial FP64 CPU oracle (test infrastructure only; see
 * zm_oracle.c for the equations and their sources in the paper).  Not included by, linked
 * into or called from the CUDA library.
 */
#ifndef ZM_ORACLE_H
#define ZM_ORACLE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ZMO_ORDER_LOW = 0, ZMO_ORDER_MEDIUM = 1, ZMO_ORDER_HIGH = 2 };

typedef struct {
    int n1, n2;      /* nodes along alpha1 (slow index) and alpha2 (fast index) */
    double L1, L2;   /* parameter-domain lengths; dx_l = L_l / n_l              */
    int periodic;    /* 1: periodic ghosts with seam shift; 0: free edges       */
} zmo_mesh;

typedef struct {
    double atwood, g, mu, delta;
    int order;       /* ZMO_ORDER_LOW, ZMO_ORDER_MEDIUM or ZMO_ORDER_HIGH */
    double cutoff;   /* > 0: Birkhoff-Rott sum over sources within this distance only */
} zmo_params;

/* All field arrays are component-major: f[c * n1 * n2 + i * n2 + j]. */
void zmo_diff1(const zmo_mesh *m, const double *f, double shift, int axis, double *out);
void zmo_laplacian(const zmo_mesh *m, const double *f, double *out);
void zmo_geometry(const zmo_mesh *m, const double *z, double *a1, double *a2, double *h,
                  double *nrm);
void zmo_sheet_strength(size_t N, const double *w, const double *a1, const double *a2,
                        double *gamma);
void zmo_br_velocity(size_t nt, const double *zt, size_t ns, const double *zs,
                     const double *gamma, double weight, double delta, double *u);
void zmo_br_velocity_cutoff(size_t nt, const double *zt, size_t ns, const double *zs,
                            const double *gamma, double weight, double delta, double cutoff,
                            double *u);
int zmo_within_cutoff(const double *zi, size_t si, const double *zj, size_t sj, double cutoff);
void zmo_fft2(int n1, int n2, double *re, double *im, int sign);
void zmo_riesz_scalar(const zmo_mesh *m, const double *w, double *s);
void zmo_phi(size_t N, const double *z, const double *w, const double *h, const double *u,
             double g, double *phi);
void zmo_wdot(const zmo_mesh *m, const double *phi, const double *w, double atwood, double mu,
              double *wdot);
int zmo_derivative(const zmo_mesh *m, const zmo_params *prm, const double *z, const double *w,
                   double *u, double *wdot);
int zmo_rk3_step(const zmo_mesh *m, const zmo_params *prm, double *z, double *w, double dt);
int zmo_run(const zmo_mesh *m, const zmo_params *prm, double *z, double *w, double dt,
            int nsteps);

#ifdef __cplusplus
}
#endif

#endif
