/*
 * oracle.c -- plain double-precision CPU oracle for the Gaussian-sum method of
 * L. Exl, N. J. Mauser and Y. Zhang, "Accurate and efficient computation of
 * nonlocal potentials based on Gaussian-sum approximation" (arXiv:1501.04438).
 *
 * TEST INFRASTRUCTURE ONLY.  It is called by the tests, by the smoke check of
 * the package entry file and by the CPU-baseline leg of the benchmark.  The
 * product (the CUDA library) never links, loads or calls it, and the two share
 * no code: not a kernel, a header, a helper, a table or a constant generator.
 *
 * The code is slow on purpose.  It is organised around the quantities the
 * paper defines, each computed from its own equation:
 *
 * Kernels: 1/(4 pi |x|) and 1/(2 pi |x|) (Coulomb), -ln|x|/(2 pi) (Poisson),
 * the dipolar and Davey-Stewartson potentials built on them (Sec. 2.4), and
 * |x|^-beta, 0 < beta < d (remark after Eq. sinc_quad).
 *
 *   quantities fixed by the kernel and the grid ("precomputation" in Algorithm 1)
 *     - Gaussian sum (w_q, tau_q) of the kernel by sinc quadrature (Sec. 3.1-3.3)
 *     - Fourier coefficients sum_q w_q G_k^q of U_GS               (Eq. tensor)
 *     - Taylor coefficients c0, c2 of the near-field ball          (Eq. taylor)
 *   quantities of one density ("actual computation" in Algorithm 1)
 *     - rho_hat by the trapezoidal rule, through an FFT            (Eq. rho_hat)
 *     - the regular part I_1, an inverse FFT of rho_hat times the
 *       stored coefficients                                        (Eq. I1FFT)
 *     - the spectral Laplacian of rho and the near-field part
 *       I_{2,1} = c0 rho + c2 Lap(rho)                             (Eq. I_2h)
 *     - u = I_1 + I_{2,1}, rescaled to the box                     (Eq. rescale)
 *
 * Every routine below is pinned by a CPU test against something other than
 * itself (closed forms, exact special cases, brute force, an independent
 * library).  No routine here is "parity unpinned".
 *
 * Conventions (readings of the paper, all double precision):
 *   - Arrays are C-ordered with x fastest: rho[z][y][x] (3D), rho[y][x] (2D).
 *   - Grid of Sec. 2.1: x_j = -L + j h, h = 2L/n, j = 1..n; array index i = j-1.
 *   - Unit-box coordinates x~ = x/L (Eq. rescale); delta is given in them.
 *     A rectangular box [-L_a, L_a] per axis (Sec. 2.5, Eq. tensor_ani and
 *     the remark after it) is rescaled by the largest half-width, L = max L_a:
 *     axis a then spans [-eta_a, eta_a], eta_a = L_a / L <= 1, its kernel box
 *     is [-2 eta_a, 2 eta_a] and its padded period 4 eta_a (6 eta_a for pad 3).
 *   - Padding factor 2 (remark after Eq. tensor: period 4) or 3 (Eq. FourSeriB3:
 *     period 6).  The kernel box of Eq. tensor is [-2,2]^d in both cases.
 *   - The GS must hold on [delta, 2 sqrt(d)]: for x in B_1 the density rho(x-y)
 *     is nonzero for y anywhere in the box B_2, whose corners lie at |y| = 2 sqrt(d).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"

#define PI 3.14159265358979323846264338327950288
#define SQRT_PI 1.77245385090551602729816748334114518

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1,1], nodes by Newton's method on the three-term */
/* recurrence of the Legendre polynomials.  (Stand-in for the Gauss-Kronrod  */
/* rule that the paper uses for Eq. tensor: any rule exact to machine        */
/* precision for these analytic integrands computes the same numbers.)       */
/* ------------------------------------------------------------------------ */
void orc_gauss_legendre(int m, double *x, double *w)
{
    for (int i = 0; i < (m + 1) / 2; i++) {
        double z = cos(PI * (i + 0.75) / (m + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= m; j++) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_m(z), p0 = P_{m-1}(z) */
            dp = m * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        /* recompute the derivative at the converged node */
        {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= m; j++) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = m * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = -z;
        x[m - 1 - i] = z;
        w[i] = w[m - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

#define GL_M 20
typedef struct { double x[GL_M], w[GL_M]; } gl_rule;

static void gl_init(gl_rule *g) { orc_gauss_legendre(GL_M, g->x, g->w); }

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: GS of 1/r.  1/r = (2/sqrt(pi)) int_0^inf exp(-r^2 tau^2) dtau    */
/* (Eq. GauInte); with tau = sinh(t) the integrand over the whole real line  */
/* is even and decays double-exponentially, and the truncated sinc rule of   */
/* Sec. 3.1 (Eq. sinc_int, 2S+1 nodes t_k = k*theta) folds to S+1 terms.     */
/* Step theta = c0 ln(S)/S with c0 = 2.1 (remark after Prop. 1).            */
/* ------------------------------------------------------------------------ */
static int gs_coulomb(int S, double c0, double *w, double *tau)
{
    double th = c0 * log((double)S) / S;
    /* 1/r = (1/sqrt(pi)) int_R exp(-r^2 sinh^2 t) cosh t dt */
    w[0] = th / SQRT_PI;          /* node t = 0: cosh 0 = 1, sinh 0 = 0 */
    tau[0] = 0.0;
    for (int k = 1; k <= S; k++) {
        double t = k * th;
        w[k] = 2.0 * th * cosh(t) / SQRT_PI;   /* nodes +t and -t folded */
        tau[k] = sinh(t);
    }
    return S + 1;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3: GS of ln r on [delta, rmax].  The paper builds a GS of 1/r^2 on  */
/* [1, R] from Eq. 1r_int with tau = ln(1 + exp(sinh t)) and moves it to     */
/* [delta, 2] by scaling.  The printed path integral for ln r is garbled; we */
/* use the equivalent Frullani form, which integrates the same 1/r^2 Gaussian */
/* representation in r and gives the same terms:                            */
/*   ln(r/delta) = 1/2 int_0^inf (e^{-t} - e^{-(r/delta)^2 t}) / t dt,        */
/* substitute t = ln(1 + e^{sinh s}) and apply the sinc rule (c0 = 1, 2S+1  */
/* nodes s_k = k*theta, k = -S..S):                                         */
/*   ln r ~ ln(delta) + C0 - sum_k wt_k exp(-t_k r^2 / delta^2),             */
/*   wt_k = theta t'(s_k) / (2 t(s_k)),  C0 = sum_k wt_k e^{-t_k}.            */
/* In the notation of Eq. log_approx: w_0 = ln(delta) + C0, tau_0 = 0, and   */
/* w_q = -wt_q, tau_q = sqrt(t_q)/delta.  t and t'/t are computed stably    */
/* for both tails, as the paper asks.                                        */
/* ------------------------------------------------------------------------ */
static void log_node(double s, double *t, double *tp_over_t)
{
    double x = sinh(s);
    double sig = 1.0 / (1.0 + exp(-x));          /* e^x / (1 + e^x) */
    double tt;
    if (x < -30.0) {
        /* t = ln(1 + e^x) = e^x (1 - e^x/2 + ...); t'/t = cosh(s) sig / t */
        double ex = exp(x);
        tt = ex * (1.0 - 0.5 * ex);
        *t = tt;
        *tp_over_t = cosh(s) * (1.0 / (1.0 + ex)) / (1.0 - 0.5 * ex);
        return;
    }
    if (x > 40.0)
        tt = x + log1p(exp(-x));
    else
        tt = log1p(exp(x));
    *t = tt;
    *tp_over_t = cosh(s) * sig / tt;
}

static int gs_log(int S, double delta, double *w, double *tau)
{
    double th = log((double)S) / S;
    double C0 = 0.0;
    int q = 1;
    for (int k = -S; k <= S; k++) {
        double t, tpt;
        log_node(k * th, &t, &tpt);
        double wt = 0.5 * th * tpt;
        C0 += wt * exp(-t);
        w[q] = -wt;
        tau[q] = sqrt(t) / delta;
        q++;
    }
    w[0] = log(delta) + C0;
    tau[0] = 0.0;
    return q;   /* 2S + 2 terms */
}

/* ------------------------------------------------------------------------ */
/* Remark after Eq. sinc_quad: GS of r^{-beta}, 0 < beta < d.  Eq. Gauss_int  */
/* with alpha = beta - 1 and rho = r^2 (the identity needs a factor 1/2 on   */
/* its right side: alpha = 0 must give Eq. GauInte) reads                    */
/*   r^{-beta} = (2/Gamma(beta/2)) int_0^inf tau^{beta-1} exp(-r^2 tau^2) dtau. */
/* The change of variables is left open.  tau = sinh t of Sec. 3.2 leaves    */
/* |sinh t|^{beta-1}, not analytic at t = 0 unless beta is odd; we take the  */
/* double-exponential map tau = exp(s - e^{-s}) (the transformation of       */
/* Takahashi and Mori for half-infinite integrals), under which              */
/*   r^{-beta} = (2/Gamma(beta/2)) int_R tau^beta (1 + e^{-s}) e^{-r^2 tau^2} ds */
/* decays double-exponentially at both ends, and apply the sinc rule of     */
/* Sec. 3.1 with S+1 nodes s_k = s_lo + k (s_hi - s_lo)/S.  The ends leave    */
/* tails below eps/4 relative to r^{-beta} on [delta, rmax]:                 */
/*   left:  (2/Gamma(beta/2)) tau_lo^beta / beta = (eps/4) rmax^{-beta}       */
/*          (the integrand is below tau^{beta-1});                           */
/*   right: delta^2 tau_hi^2 = ln(1/eps) + 10, where the relative tail is    */
/*          the regularised Q(beta/2, delta^2 tau_hi^2) < e^{-10} eps/4 (beta < 3); */
/* s_lo and s_hi solve s - e^{-s} = ln tau by Newton's method, started left */
/* of the root (the map is concave, so the iterates increase to it).         */
/* ------------------------------------------------------------------------ */
static double de_solve(double X)
{
    double s = X > -1.0 ? X - 1.0 : -log(-X);
    for (int it = 0; it < 100; it++) {
        double ds = (s - exp(-s) - X) / (1.0 + exp(-s));
        s -= ds;
        if (fabs(ds) <= 1e-15 * (1.0 + fabs(s))) break;
    }
    return s;
}

static void power_ends(double beta, double delta, double rmax, double eps, double *slo, double *shi)
{
    double cn = 2.0 / tgamma(0.5 * beta);
    double ln_tau_lo = (log(0.25 * eps * beta / cn) - beta * log(rmax)) / beta;
    double ln_tau_hi = 0.5 * log(log(1.0 / eps) + 10.0) - log(delta);
    *slo = de_solve(ln_tau_lo);
    *shi = de_solve(ln_tau_hi);
}

static int gs_power(int S, double beta, double delta, double rmax, double eps, double *w, double *tau)
{
    double slo, shi;
    power_ends(beta, delta, rmax, eps, &slo, &shi);
    double th = (shi - slo) / S, cn = 2.0 / tgamma(0.5 * beta);
    for (int k = 0; k <= S; k++) {
        double s = slo + k * th;
        double lt = s - exp(-s);               /* ln tau */
        tau[k] = exp(lt);
        w[k] = cn * th * exp(beta * lt) * (1.0 + exp(-s));
    }
    return S + 1;
}

double orc_gs_eval(int nterms, const double *w, const double *tau, double r)
{
    double s = 0.0;
    for (int q = 0; q < nterms; q++) {
        double a = tau[q] * r;
        s += w[q] * exp(-a * a);
    }
    return s;
}

static int kernel_is_log(int kernel) { return kernel == ORC_POISSON_2D; }
static int kernel_is_power(int kernel) { return kernel == ORC_POWER_3D || kernel == ORC_POWER_2D; }

/* E_rel (1/r, Sec. 3.2; r^{-beta}) or E_abs (ln r, Sec. 3.3) on a geometric */
/* sample of [delta, rmax] with ns points, both end points included.         */
double orc_gs_error(int kernel, double beta, int nterms, const double *w, const double *tau,
                    double delta, double rmax, int ns)
{
    double e = 0.0;
    for (int i = 0; i < ns; i++) {
        double r = delta * pow(rmax / delta, (double)i / (ns - 1));
        double g = orc_gs_eval(nterms, w, tau, r);
        double err;
        if (kernel_is_log(kernel)) err = fabs(log(r) - g);
        else if (kernel_is_power(kernel)) err = fabs(1.0 - pow(r, beta) * g);
        else err = fabs(1.0 - r * g);
        if (err > e) e = err;
    }
    return e;
}

int orc_gs_build(int kernel, double beta, double delta, double rmax, double eps, int S_fixed,
                 int cap, double *w, double *tau, int *nterms, int *S_out, double *err)
{
    int Smin = S_fixed > 0 ? S_fixed : 4;
    int Smax = S_fixed > 0 ? S_fixed : ORC_GS_SMAX;
    for (int S = Smin; S <= Smax; S++) {
        int need = kernel_is_log(kernel) ? 2 * S + 2 : S + 1;
        if (need > cap) return ORC_ERR;
        int nt;
        if (kernel_is_log(kernel)) nt = gs_log(S, delta, w, tau);
        else if (kernel_is_power(kernel)) nt = gs_power(S, beta, delta, rmax, eps, w, tau);
        else nt = gs_coulomb(S, 2.1, w, tau);
        double e = orc_gs_error(kernel, beta, nt, w, tau, delta, rmax, ORC_GS_NSAMPLE);
        if (S_fixed > 0 || e <= eps) {
            *nterms = nt;
            *S_out = S;
            *err = e;
            return ORC_OK;
        }
    }
    return ORC_ERR;
}

/* ------------------------------------------------------------------------ */
/* Eq. tensor: one 1-D factor                                                */
/*   g(tau, omega) = int_{-2}^{2} exp(-tau^2 y^2) cos(omega y) dy,            */
/* omega = 2 pi k / P.  Composite 20-point Gauss-Legendre on [0, b], b = 2,  */
/* or b = 7/tau when that is smaller (the integrand is below e^{-49} there). */
/* Panels are short enough to resolve both the Gaussian and the cosine.     */
/* ------------------------------------------------------------------------ */
static double factor_gl(const gl_rule *g, double tau, double omega, double half)
{
    double b = half;   /* integrate over [0, half], half = 2 eta */
    if (tau > 0.0 && 7.0 / tau < b) b = 7.0 / tau;
    double scale = tau > fabs(omega) ? tau : fabs(omega);
    int np = 2 + (int)ceil(b * scale / 2.0);
    double hb = b / np, sum = 0.0;
    for (int p = 0; p < np; p++) {
        double mid = (p + 0.5) * hb, ps = 0.0;
        for (int j = 0; j < GL_M; j++) {
            double y = mid + 0.5 * hb * g->x[j];
            ps += g->w[j] * exp(-(tau * y) * (tau * y)) * cos(omega * y);
        }
        sum += 0.5 * hb * ps;
    }
    return 2.0 * sum;
}

double orc_factor(double tau, double omega)
{
    gl_rule g;
    gl_init(&g);
    return factor_gl(&g, tau, omega, 2.0);
}

/* ------------------------------------------------------------------------ */
/* FFT used by the oracle: recursive mixed-radix decimation in time.         */
/*   out[k] = sum_j in[j*stride] exp(sign * 2 pi i j k / n)   (unnormalised)  */
/* At each level the length is split by its smallest prime factor p; the p   */
/* sub-transforms are combined with an explicit p-point DFT.  Twiddles come  */
/* from a table e^{sign 2 pi i j / N} of the top-level length N.             */
/* ------------------------------------------------------------------------ */
static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

static void fft_rec(const cplx *in, size_t stride, cplx *out, int n,
                    const cplx *tw, int N, cplx *scratch)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = smallest_factor(n), m = n / p;
    for (int r = 0; r < p; r++)
        fft_rec(in + r * stride, stride * p, out + (size_t)r * m, m, tw, N, scratch);
    /* X[k + s m] = sum_r e^{sign 2 pi i r (k + s m) / n} Y_r[k] */
    int step = N / n;
    for (int k = 0; k < m; k++)
        for (int s = 0; s < p; s++) {
            cplx acc = 0.0;
            for (int r = 0; r < p; r++) {
                long e = ((long)r * (k + (long)s * m)) % n;
                acc += tw[e * step] * out[(size_t)r * m + k];
            }
            scratch[k + s * m] = acc;
        }
    memcpy(out, scratch, sizeof(cplx) * n);
}

static cplx *twiddle_table(int N, int sign)
{
    cplx *tw = malloc(sizeof(cplx) * N);
    for (int j = 0; j < N; j++) {
        double a = 2.0 * PI * (double)j / N;
        tw[j] = cos(a) + sign * sin(a) * I;
    }
    return tw;
}

/* In-place unnormalised DFT along every axis of a C-ordered array whose     */
/* extents are shape[0] (fastest, x), shape[1], shape[2].                    */
int orc_fftn(int d, const int *shape, double *data, int sign)
{
    cplx *a = (cplx *)data;
    size_t total = 1;
    for (int i = 0; i < d; i++) total *= (size_t)shape[i];
    size_t stride = 1;
    for (int ax = 0; ax < d; ax++) {
        int N = shape[ax];
        cplx *tw = twiddle_table(N, sign);
        size_t nlines = total / N;
#pragma omp parallel
        {
            cplx *line = malloc(sizeof(cplx) * N);
            cplx *res = malloc(sizeof(cplx) * N);
            cplx *scr = malloc(sizeof(cplx) * N);
#pragma omp for schedule(static)
            for (long l = 0; l < (long)nlines; l++) {
                size_t inner = (size_t)l % stride, outer = (size_t)l / stride;
                size_t base = outer * stride * N + inner;
                for (int j = 0; j < N; j++) line[j] = a[base + (size_t)j * stride];
                fft_rec(line, 1, res, N, tw, N, scr);
                for (int j = 0; j < N; j++) a[base + (size_t)j * stride] = res[j];
            }
            free(line);
            free(res);
            free(scr);
        }
        free(tw);
        stride *= (size_t)N;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3: near-field correction coefficients.  With the Taylor polynomial */
/* of Eq. taylor, odd terms and off-diagonal second derivatives integrate to */
/* zero over the ball B_delta, and the sphere average of y_j^2 is r^2/d, so   */
/*   I_{2,1} ~ c0 rho + c2 Lap(rho),                                          */
/*   c0 = |S^{d-1}| A_{d-1},  c2 = |S^{d-1}| / (2d) A_{d+1},                   */
/*   A_m = int_0^delta r^m (U1(r) - U_GS(r)) dr,                              */
/* with U1 = 1/r (Coulomb) or ln r (Poisson; the factor -1/(2 pi) and the     */
/* rescaling constants are applied outside).  The U1 part is integrated      */
/* exactly; the Gaussian part by composite Gauss-Legendre.                   */
/* ------------------------------------------------------------------------ */
static double gauss_moment(const gl_rule *g, int m, double tau, double delta)
{
    /* int_0^delta r^m exp(-tau^2 r^2) dr */
    if (tau == 0.0) return pow(delta, m + 1) / (m + 1);
    double b = delta;
    if (9.0 / tau < b) b = 9.0 / tau;
    int np = 2 + (int)ceil(b * tau / 2.0);
    double hb = b / np, sum = 0.0;
    for (int p = 0; p < np; p++) {
        double mid = (p + 0.5) * hb, ps = 0.0;
        for (int j = 0; j < GL_M; j++) {
            double r = mid + 0.5 * hb * g->x[j];
            ps += g->w[j] * pow(r, m) * exp(-(tau * r) * (tau * r));
        }
        sum += 0.5 * hb * ps;
    }
    return sum;
}

static double kernel_moment(int kernel, double beta, int m, double delta)
{
    /* int_0^delta r^m U1(r) dr */
    if (kernel_is_log(kernel))
        return pow(delta, m + 1) * (log(delta) / (m + 1) - 1.0 / ((m + 1.0) * (m + 1.0)));
    if (kernel_is_power(kernel))
        return pow(delta, m + 1 - beta) / (m + 1 - beta);   /* U1 = r^{-beta}, beta < m + 1 */
    return pow(delta, m) / m;   /* U1 = 1/r */
}

int orc_taylor_coeffs(int kernel, double beta, int d, int nterms, const double *w, const double *tau,
                      double delta, double *c0, double *c2)
{
    gl_rule g;
    gl_init(&g);
    double area = (d == 3) ? 4.0 * PI : 2.0 * PI;   /* |S^{d-1}| */
    double A[2];
    int ms[2] = {d - 1, d + 1};
    for (int i = 0; i < 2; i++) {
        double gs = 0.0;
        for (int q = 0; q < nterms; q++) gs += w[q] * gauss_moment(&g, ms[i], tau[q], delta);
        A[i] = kernel_moment(kernel, beta, ms[i], delta) - gs;
    }
    *c0 = area * A[0];
    *c2 = area / (2.0 * d) * A[1];
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Whole evaluation.                                                         */
/* ------------------------------------------------------------------------ */
static int base_kernel(int kernel)
{
    /* The dipolar potential is a 3D Coulomb potential of d_nm rho (Sec. 2.4); */
    /* the Davey-Stewartson potential a 2D Poisson potential of d_xx rho       */
    /* (end of Sec. 2.4, Example 5).                                          */
    if (kernel == ORC_DIPOLAR_3D) return ORC_COULOMB_3D;
    if (kernel == ORC_DS_2D) return ORC_POISSON_2D;
    return kernel;
}

static int kernel_dim(int kernel)
{
    return (kernel == ORC_COULOMB_3D || kernel == ORC_DIPOLAR_3D || kernel == ORC_POWER_3D) ? 3 : 2;
}

static size_t prod(int d, const int *n)
{
    size_t t = 1;
    for (int i = 0; i < d; i++) t *= (size_t)n[i];
    return t;
}

/* sum of a[0..n) by recursive halving: rounding error O(eps log n) */
static double pairwise_sum(const double *a, size_t n)
{
    if (n <= 16) {
        double s = 0.0;
        for (size_t i = 0; i < n; i++) s += a[i];
        return s;
    }
    return pairwise_sum(a, n / 2) + pairwise_sum(a + n / 2, n - n / 2);
}

/* signed frequency of DFT index j of length N: j or j - N */
static int signed_freq(int j, int N) { return j < (N + 1) / 2 ? j : j - N; }

/* Reference half-width Lr and per-axis eta_a of Sec. 2.5 (all 1 for the     */
/* cubic box [-L, L]^d).                                                     */
static double box_eta(const orc_params_t *p, double *eta)
{
    int d = kernel_dim(p->kernel);
    double Lr = 0.0;
    for (int a = 0; a < d; a++)
        if (p->box[a] > Lr) Lr = p->box[a];
    if (Lr <= 0.0) {
        for (int a = 0; a < 3; a++) eta[a] = 1.0;
        return p->L;
    }
    for (int a = 0; a < 3; a++) eta[a] = a < d ? p->box[a] / Lr : 1.0;
    return Lr;
}

int orc_plan_gs(const orc_params_t *p, double *w, double *tau, int cap, orc_info_t *info)
{
    int kb = base_kernel(p->kernel);
    int d = kernel_dim(p->kernel);
    double eta[3];
    box_eta(p, eta);
    double rr = 0.0;   /* the kernel box B_2 (per axis [-2 eta, 2 eta]) has its corners at 2|eta| */
    for (int a = 0; a < d; a++) rr += eta[a] * eta[a];
    double rmax = 2.0 * sqrt(rr);
    int nt, S;
    double err;
    if (orc_gs_build(kb, p->beta, p->delta, rmax, p->gs_eps, p->gs_S, cap, w, tau, &nt, &S, &err) != ORC_OK)
        return -1;   /* no Gaussian sum meets gs_eps (callers test nt <= 0) */
    if (info) {
        info->S = S;
        info->nterms = nt;
        info->gs_err = err;
    }
    return nt;
}

/* Octant of sum_q w_q G_k^q (Eq. tensor) for k_j = 0..Nt_j/2, Nt = pad*n.   */
/* Layout [kz][ky][kx] (3D) or [ky][kx] (2D), kx fastest.                    */
int orc_kernel_hat(const orc_params_t *p, double *khat, orc_info_t *info)
{
    int d = kernel_dim(p->kernel);
    double w[ORC_GS_CAP], tau[ORC_GS_CAP];
    int nt = orc_plan_gs(p, w, tau, ORC_GS_CAP, info);
    if (nt <= 0) return ORC_ERR;
    double eta[3];
    box_eta(p, eta);
    int no[3] = {1, 1, 1};
    for (int a = 0; a < d; a++) no[a] = p->pad * p->n[a] / 2 + 1;
    /* 1-D factors per axis: g[a][q][k] */
    double *g[3] = {NULL, NULL, NULL};
    gl_rule gl;
    gl_init(&gl);
    for (int a = 0; a < d; a++) {
        g[a] = malloc(sizeof(double) * nt * no[a]);
#pragma omp parallel for collapse(2) schedule(dynamic)
        for (int q = 0; q < nt; q++)
            for (int k = 0; k < no[a]; k++)
                g[a][(size_t)q * no[a] + k] =
                    factor_gl(&gl, tau[q], 2.0 * PI * k / (2.0 * p->pad * eta[a]), 2.0 * eta[a]);
    }
    size_t tot = (size_t)no[0] * no[1] * no[2];
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < (long)tot; idx++) {
        int kx = idx % no[0], ky = (idx / no[0]) % no[1], kz = idx / ((size_t)no[0] * no[1]);
        double s = 0.0;
        for (int q = 0; q < nt; q++) {
            double t = w[q] * g[0][(size_t)q * no[0] + kx] * g[1][(size_t)q * no[1] + ky];
            if (d == 3) t *= g[2][(size_t)q * no[2] + kz];
            s += t;
        }
        khat[idx] = s;
    }
    for (int a = 0; a < d; a++) free(g[a]);
    return ORC_OK;
}

/* Laplacian (unit-box coordinates) or the d_nm derivative (physical        */
/* coordinates) of rho on the n-grid by FFT, period 2 in unit coordinates.  */
/* which = 0: Laplacian; which = 1: d_nm = sum_ij n_i m_j d_i d_j.            */
static void spectral_derivative(int d, const int *n, double L, const double *eta, int which,
                                const double *dn, const double *dm,
                                const double *rho, double *out)
{
    size_t N = prod(d, n);
    cplx *a = malloc(sizeof(cplx) * N);
    for (size_t i = 0; i < N; i++) a[i] = rho[i];
    orc_fftn(d, n, (double *)a, -1);
    int nn[3] = {n[0], d > 1 ? n[1] : 1, d > 2 ? n[2] : 1};
    for (size_t idx = 0; idx < N; idx++) {
        int k[3] = {(int)(idx % nn[0]), (int)((idx / nn[0]) % nn[1]), (int)(idx / ((size_t)nn[0] * nn[1]))};
        double kap[3] = {0, 0, 0};
        int nyq[3] = {0, 0, 0};
        for (int j = 0; j < d; j++) {
            int f = signed_freq(k[j], n[j]);
            nyq[j] = (2 * f == -n[j]);
            kap[j] = PI * f / eta[j];     /* 2 pi f / period, period 2 eta_j */
        }
        double mult;
        if (which == 0) {
            mult = 0.0;
            for (int j = 0; j < d; j++) mult -= kap[j] * kap[j];
        } else {
            /* (i n.kappa)(i m.kappa); first derivatives vanish at Nyquist */
            mult = 0.0;
            for (int i = 0; i < d; i++)
                for (int j = 0; j < d; j++) {
                    if (i != j && (nyq[i] || nyq[j])) continue;
                    mult -= dn[i] * dm[j] * kap[i] * kap[j] / (L * L);
                }
        }
        a[idx] *= mult;
    }
    orc_fftn(d, n, (double *)a, +1);
    for (size_t i = 0; i < N; i++) out[i] = creal(a[i]) / (double)N;
    free(a);
}

/* Precomputation of Algorithm 1 for one scalar potential (Coulomb 3D/2D or */
/* Poisson 2D): Gaussian sum, Taylor coefficients and the octant of         */
/* sum_q w_q G^q_k.  Kept apart from the actual computation so that the two  */
/* can be timed separately, as the paper does.                              */
struct orc_prepared_s {
    orc_params_t p;
    int kernel, d;
    double c0, c2;
    double *khat;
    int Nt[3], no[3];
    orc_info_t info;
};

static struct orc_prepared_s *prepare_scalar(const orc_params_t *p, int kernel)
{
    struct orc_prepared_s *h = calloc(1, sizeof(*h));
    h->p = *p;
    h->p.kernel = kernel;
    h->kernel = kernel;
    h->d = kernel_dim(kernel);
    double w[ORC_GS_CAP], tau[ORC_GS_CAP];
    int nt = orc_plan_gs(&h->p, w, tau, ORC_GS_CAP, &h->info);
    if (nt <= 0) {
        free(h);
        return NULL;
    }
    orc_taylor_coeffs(kernel, p->beta, h->d, nt, w, tau, p->delta, &h->c0, &h->c2);
    h->info.c0 = h->c0;
    h->info.c2 = h->c2;
    for (int a = 0; a < 3; a++) {
        h->Nt[a] = a < h->d ? p->pad * p->n[a] : 1;
        h->no[a] = a < h->d ? h->Nt[a] / 2 + 1 : 1;
    }
    h->khat = malloc(sizeof(double) * h->no[0] * h->no[1] * h->no[2]);
    if (orc_kernel_hat(&h->p, h->khat, NULL) != ORC_OK) {
        free(h->khat);
        free(h);
        return NULL;
    }
    return h;
}

/* Actual computation of Algorithm 1 for one scalar potential.               */
/* dn, dm non-NULL (taylor_mode 1 only): the source is d_nm rho, applied as  */
/* the symbol -(n.kappa)(m.kappa) of the padded grid (physical units).       */
static int run_scalar(const struct orc_prepared_s *h, const double *rho, double *u,
                      double *i1_out, double *i2_out, const double *dn, const double *dm)
{
    const orc_params_t *p = &h->p;
    const int kernel = h->kernel, d = h->d;
    const int *n = p->n;
    const int *Nt = h->Nt, *no = h->no;
    double eta[3];
    const double L = box_eta(p, eta), c0 = h->c0, c2 = h->c2;
    const double *khat = h->khat;

    /* rho_hat: zero-padded density, rho_hat_k = DFT / Nt^d (Eq. rho_hat,    */
    /* trapezoidal rule).  Grid point i sits at padded index i + off with    */
    /* off = 1 + (pad - 1) n / 2 (periodic box [-P/2, P/2), P = 2 pad).       */
    size_t NT = prod(d, Nt), N = prod(d, n);
    cplx *a = calloc(NT, sizeof(cplx));
    int off[3];
    for (int j = 0; j < 3; j++) off[j] = j < d ? 1 + (p->pad - 1) * n[j] / 2 : 0;
    int n3[3] = {n[0], d > 1 ? n[1] : 1, d > 2 ? n[2] : 1};
    for (size_t i = 0; i < N; i++) {
        int x = i % n3[0], y = (i / n3[0]) % n3[1], z = i / ((size_t)n3[0] * n3[1]);
        size_t m = (size_t)(x + off[0]) + (size_t)Nt[0] * ((y + off[1]) + (size_t)Nt[1] * (z + off[2]));
        a[m] = rho[i];
    }
    orc_fftn(d, Nt, (double *)a, -1);
    double invN = 1.0 / (double)NT;

    /* I_1(x) = sum_k rho_hat_k (sum_q w_q G^q_k) e^{2 pi i k (x - a)/P}        */
    /* (Eq. I1FFT).  taylor_mode 1 also folds c0 - c2 |kappa|^2 into the     */
    /* multiplier: the Taylor correction with a padded-grid spectral Laplacian. */
    /* Period of axis j: P_j = 2 pad eta_j.                                   */
    double P[3];
    for (int j = 0; j < 3; j++) P[j] = 2.0 * p->pad * eta[j];
    for (size_t idx = 0; idx < NT; idx++) {
        int k[3] = {(int)(idx % Nt[0]), (int)((idx / Nt[0]) % Nt[1]), (int)(idx / ((size_t)Nt[0] * Nt[1]))};
        int kk[3] = {0, 0, 0};
        double kap2 = 0.0;
        for (int j = 0; j < d; j++) {
            int f = signed_freq(k[j], Nt[j]);
            kk[j] = abs(f);
            double kap = 2.0 * PI * f / P[j];
            kap2 += kap * kap;
        }
        double mult = khat[kk[0] + (size_t)no[0] * (kk[1] + (size_t)no[1] * kk[2])];
        if (p->taylor_mode == 1) mult += c0 - c2 * kap2;
        if (dn) {
            /* -(n.kappa)(m.kappa) / L^2; first derivatives vanish at Nyquist */
            double kv[3] = {0, 0, 0}, sym = 0.0;
            int nyq[3] = {0, 0, 0};
            for (int j = 0; j < d; j++) {
                int f = signed_freq(k[j], Nt[j]);
                kv[j] = 2.0 * PI * f / P[j];
                nyq[j] = (2 * f == -Nt[j]);
            }
            for (int i = 0; i < d; i++)
                for (int j = 0; j < d; j++) {
                    if (i != j && (nyq[i] || nyq[j])) continue;
                    sym -= dn[i] * dm[j] * kv[i] * kv[j] / (L * L);
                }
            mult *= sym;
        }
        a[idx] *= mult * invN;
    }
    orc_fftn(d, Nt, (double *)a, +1);

    /* Lap(rho) on the n-grid (spectral), for the literal near-field part */
    double *lap = NULL;
    if (p->taylor_mode == 0) {
        lap = malloc(sizeof(double) * N);
        spectral_derivative(d, n, L, eta, 0, NULL, NULL, rho, lap);
    }

    /* Rescaling of Sec. 2.1 (Eq. rescale and the two lines after it) */
    double s;
    if (kernel == ORC_COULOMB_3D) s = L * L / (4.0 * PI);
    else if (kernel == ORC_COULOMB_2D) s = L / (2.0 * PI);
    else if (kernel_is_power(kernel)) s = pow(L, d - p->beta);   /* |L x~|^{-beta} L^d dx~ */
    else s = -L * L / (2.0 * PI);              /* ln kernel, -1/(2 pi) ln|x| */
    double extra = 0.0;
    if (kernel == ORC_POISSON_2D && !dn) {   /* a derivative source has zero mass */
        /* trapezoidal int rho~, summed pairwise (a sequential sum over n^2    */
        /* points drifts by ~1e-12 relative at n = 4096)                       */
        double hu = 2.0 * eta[0] / n[0], hv = 2.0 * eta[1] / n[1];
        double mass = pairwise_sum(rho, N);
        extra = -L * L / (2.0 * PI) * log(L) * hu * hv * mass;
    }

    /* I_{2,1} ~ c0 rho + c2 Lap(rho) (Eq. I_2h) and u = I_1 + I_{2,1}        */
    for (size_t i = 0; i < N; i++) {
        int x = i % n3[0], y = (i / n3[0]) % n3[1], z = i / ((size_t)n3[0] * n3[1]);
        size_t m = (size_t)(x + off[0]) + (size_t)Nt[0] * ((y + off[1]) + (size_t)Nt[1] * (z + off[2]));
        double i1 = creal(a[m]);
        double i2 = (p->taylor_mode == 0) ? c0 * rho[i] + c2 * lap[i] : 0.0;
        if (i1_out) i1_out[i] = s * i1;
        if (i2_out) i2_out[i] = s * i2;
        u[i] = s * (i1 + i2) + extra;
    }
    free(lap);
    free(a);
    return ORC_OK;
}

static int check_params(const orc_params_t *p)
{
    int d = kernel_dim(p->kernel);
    double eta[3];
    if (p->d != d || box_eta(p, eta) <= 0 || p->delta <= 0 || (p->pad != 2 && p->pad != 3)) return ORC_ERR;
    for (int a = 0; a < d; a++)
        if (p->delta >= eta[a]) return ORC_ERR;   /* Sec. 2.5: delta smaller than eta */
    if (kernel_is_power(p->kernel) && !(p->beta > 0.0 && p->beta < d)) return ORC_ERR;
    for (int a = 0; a < d; a++)
        if (p->n[a] < 2 || p->n[a] % 2) return ORC_ERR;
#ifdef _OPENMP
    if (p->threads > 0) omp_set_num_threads(p->threads);
#endif
    return ORC_OK;
}

orc_prepared_t *orc_prepare(const orc_params_t *p, orc_info_t *info)
{
    if (check_params(p) != ORC_OK) return NULL;
    struct orc_prepared_s *h = prepare_scalar(p, base_kernel(p->kernel));
    if (h) {
        h->p.kernel = p->kernel;      /* remember the dipolar request */
        if (info) *info = h->info;
    }
    return h;
}

void orc_free_prepared(orc_prepared_t *h)
{
    if (!h) return;
    free(h->khat);
    free(h);
}

/* Actual computation for a prepared problem (the dipolar kernel of Sec. 2.4  */
/* and Example 4: u = -(n.m) rho - 3 U_C * (d_nm rho), with d_nm rho from the */
/* Fourier pseudospectral interpolant of the n-grid (taylor_mode 0) or of the */
/* zero-padded grid (taylor_mode 1)).                                        */
int orc_run(const orc_prepared_t *h, const double *rho, double *u, double *i1, double *i2)
{
    const orc_params_t *p = &h->p;
#ifdef _OPENMP
    if (p->threads > 0) omp_set_num_threads(p->threads);
#endif
    if (p->kernel == ORC_DS_2D) {
        /* Example 5: u = -(1/2 pi) ln|x| * (d_xx rho), d_xx rho from the Fourier */
        /* interpolant of the n-grid (taylor_mode 0) or the padded grid (1)       */
        static const double ex[3] = {1.0, 0.0, 0.0};
        if (p->taylor_mode == 1) return run_scalar(h, rho, u, i1, i2, ex, ex);
        size_t N = prod(2, p->n);
        double *src = malloc(sizeof(double) * N);
        double eta[3];
        double Lr = box_eta(p, eta);
        spectral_derivative(2, p->n, Lr, eta, 1, ex, ex, rho, src);
        int rc = run_scalar(h, src, u, i1, i2, NULL, NULL);
        free(src);
        return rc;
    }
    if (p->kernel != ORC_DIPOLAR_3D) return run_scalar(h, rho, u, i1, i2, NULL, NULL);
    size_t N = prod(3, p->n);
    double *src = malloc(sizeof(double) * N), *uc = malloc(sizeof(double) * N);
    int rc;
    if (p->taylor_mode == 0) {
        double eta[3];
        double Lr = box_eta(p, eta);
        spectral_derivative(3, p->n, Lr, eta, 1, p->dip_n, p->dip_m, rho, src);
        rc = run_scalar(h, src, uc, NULL, NULL, NULL, NULL);
    } else {
        rc = run_scalar(h, rho, uc, NULL, NULL, p->dip_n, p->dip_m);
    }
    double nm = p->dip_n[0] * p->dip_m[0] + p->dip_n[1] * p->dip_m[1] + p->dip_n[2] * p->dip_m[2];
    for (size_t i = 0; i < N; i++) u[i] = -nm * rho[i] - 3.0 * uc[i];
    free(src);
    free(uc);
    return rc;
}

int orc_apply_parts(const orc_params_t *p, const double *rho, double *u,
                    double *i1, double *i2, orc_info_t *info)
{
    orc_prepared_t *h = orc_prepare(p, info);
    if (!h) return ORC_ERR;
    int rc = orc_run(h, rho, u, i1, i2);
    orc_free_prepared(h);
    return rc;
}

int orc_apply(const orc_params_t *p, const double *rho, double *u, orc_info_t *info)
{
    return orc_apply_parts(p, rho, u, NULL, NULL, info);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
