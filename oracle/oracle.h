/*
 * oracle.h -- interface of the plain FP64 CPU oracle (test infrastructure only;
 * see oracle.c).  Exl, Mauser, Zhang, arXiv:1501.04438.
 */
#ifndef GSM_ORACLE_H
#define GSM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_COULOMB_3D = 0, ORC_COULOMB_2D = 1, ORC_POISSON_2D = 2, ORC_DIPOLAR_3D = 3, ORC_DS_2D = 4,
       ORC_POWER_3D = 5, ORC_POWER_2D = 6 };   /* power: U = |x|^{-beta}, 0 < beta < d */
enum { ORC_OK = 0, ORC_ERR = 1 };

#define ORC_GS_CAP 1024      /* max number of Gaussian terms */
#define ORC_GS_SMAX 400      /* largest S tried when choosing S */
#define ORC_GS_NSAMPLE 4000  /* geometric sample of [delta, rmax] for the GS error */

typedef struct {
    int kernel;         /* ORC_* kernel */
    int d;              /* dimension, 2 or 3 */
    int n[3];           /* points per axis, x first; even */
    double L;           /* box [-L, L]^d */
    int pad;            /* 2 (period 4, default) or 3 (period 6) */
    double delta;       /* radius of the near-field ball, unit-box coordinates */
    double gs_eps;      /* GS accuracy target: E_rel (1/r) or E_abs (ln r) */
    int gs_S;           /* > 0: use this S; 0: smallest S meeting gs_eps */
    int taylor_mode;    /* 0: Laplacian on the n-grid; 1: folded, padded grid */
    double dip_n[3];    /* dipolar unit vectors n and m */
    double dip_m[3];
    int threads;        /* OpenMP threads (0: default) */
    double box[3];      /* > 0: half-width of axis a (rectangular box, Sec. 2.5); */
                        /* all 0: the cube [-L, L]^d                           */
    double beta;        /* exponent of the power kernels */
} orc_params_t;

typedef struct {
    int S, nterms;
    double gs_err, c0, c2;
} orc_info_t;

void orc_gauss_legendre(int m, double *x, double *w);
double orc_gs_eval(int nterms, const double *w, const double *tau, double r);
double orc_gs_error(int kernel, double beta, int nterms, const double *w, const double *tau,
                    double delta, double rmax, int ns);
int orc_gs_build(int kernel, double beta, double delta, double rmax, double eps, int S_fixed,
                 int cap, double *w, double *tau, int *nterms, int *S_out, double *err);
double orc_factor(double tau, double omega);
int orc_fftn(int d, const int *shape, double *data, int sign);
int orc_taylor_coeffs(int kernel, double beta, int d, int nterms, const double *w, const double *tau,
                      double delta, double *c0, double *c2);
int orc_plan_gs(const orc_params_t *p, double *w, double *tau, int cap, orc_info_t *info);
int orc_kernel_hat(const orc_params_t *p, double *khat, orc_info_t *info);
int orc_apply_parts(const orc_params_t *p, const double *rho, double *u,
                    double *i1, double *i2, orc_info_t *info);
int orc_apply(const orc_params_t *p, const double *rho, double *u, orc_info_t *info);

/* Precomputation and actual computation of Algorithm 1 kept apart. */
typedef struct orc_prepared_s orc_prepared_t;
orc_prepared_t *orc_prepare(const orc_params_t *p, orc_info_t *info);
int orc_run(const orc_prepared_t *h, const double *rho, double *u, double *i1, double *i2);
void orc_free_prepared(orc_prepared_t *h);
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
