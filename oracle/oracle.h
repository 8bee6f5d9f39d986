/* FP64 CPU oracle (test infrastructure only): declarations for oracle.c. */
#ifndef ORC_ORACLE_H
#define ORC_ORACLE_H
#include <stdint.h>

enum { ORC_CONVERGED = 0, ORC_MAXITER = 1, ORC_LS_STALLED = 2, ORC_NONFINITE = 3, ORC_ZERO_GRADIENT = 4 };

typedef struct orc_params {
    int32_t n_levels;
    int32_t iter_max;
    double epsilon;
    double lambda;
    double armijo_sigma;
    double tau_init;
    double tau_max;
    double tau_min;
    double smooth;  /* H1-type smoother width in grid spacings (0: lumped-mass L2 flow) */
} orc_params;

typedef struct orc_level_stats {
    int32_t iters;
    int32_t trials;
    int32_t status;
    int32_t pad;
    double E_start;
    double E;
    double tau;
} orc_level_stats;

void orc_set_trace(double *buf, long cap);
long orc_trace_len(void);
void orc_embed(const float *frame, int side, double *out);
void orc_restrict(const double *fine, int nf, double *coarse);
void orc_prolong(const double *coarse, int nc, double *fine);
void orc_mass_apply(const double *v, int n, double *out);
void orc_stiff_apply(const double *v, int n, double *out);
void orc_lumped(int n, double *w);
double orc_interp(const double *T, int n, double x0, double x1, double *d0, double *d1);
void orc_warp(const double *T, int n, const double *u, double *That, double *dT);
double orc_energy(const double *R, const double *T, int n, const double *u, double lambda, double *parts);
void orc_gradient(const double *R, const double *T, int n, const double *u, double lambda, double *g);
int orc_solve_level(const double *R, const double *T, int n, double *u, const orc_params *p,
                    orc_level_stats *st);
int orc_register(const double *R, const double *T, int L, const double *u_init, const orc_params *p,
                 double *u_out, orc_level_stats *st);
void orc_compose(const double *u_ij, const double *u_jk, int n, double *out);
void orc_apply_batch(int n_ops, const double *const *R, const double *const *T, const int32_t *L,
                     const double *const *left, const double *const *right, double *const *out,
                     const orc_params *p, int32_t *status, int32_t *iters, int32_t *trials,
                     double *energy);
void orc_average(int m, const double *const *F, const double *const *u, int n, double *avg);
void orc_rigid_field(const double *theta, int n, double *u);
double orc_rigid_energy(const double *R, const double *T, int n, const double *theta, double lambda);
void orc_rigid_gradient(const double *R, const double *T, int n, const double *theta, double lambda, double *grad);
int orc_rigid_solve_level(const double *R, const double *T, int n, double *theta, const orc_params *p,
                          orc_level_stats *st);
int orc_rigid_register(const double *R, const double *T, int L, const double *theta_init, const orc_params *p,
                       double *theta_out, orc_level_stats *st);
void orc_rigid_compose(const double *a, const double *b, double *out);
void orc_smooth_apply(int n, double smooth, const double *g, double *d);
void orc_smooth_matvec(int n, double smooth, const double *v, double *out);
#endif
