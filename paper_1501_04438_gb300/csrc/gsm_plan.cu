// gsm_plan.cu -- Algorithm 1, "Precomputation", on the GPU in FP64.
//
//   1. Gaussian sum U_GS(r) = sum_q w_q exp(-tau_q^2 r^2) of 1/r (Sec. 3.2),
//      ln r (Sec. 3.3) or r^-beta (remark after Eq. sinc_quad) by truncated
//      sinc quadrature (Sec. 3.1), S chosen as the smallest value whose error
//      on [delta, 2 |eta|] meets the target.
//   2. One-dimensional factors g_q(k) of Eq. tensor.
//   3. Near-field coefficients c0, c2 of Sec. 2.3.
//   4. The tensor sum_q w_q g_q(kx) g_q(ky) g_q(kz) on the octant, and the
//      multiplier applied by the passes (Taylor correction, rescaling of
//      Sec. 2.1, FFT normalisation, dipolar symbol of Sec. 2.4 folded in).
#include <math.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gsm_internal.h"

namespace gsm {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double kSqrtPi = 1.77245385090551602729816748334114518;
constexpr int kNSample = 6000;   // geometric sample of [delta, rmax] for the GS error
constexpr int kWeidN = 64;       // terms of the rational approximation of w(z)
constexpr int kTaylorJ = 44;     // terms of the small-tau series of g
constexpr double kTauSeries = 1.0;   // g by series below, by w(z) above
constexpr double kTauGauss = 4.0;    // g by the Gaussian transform at and above

__host__ __device__ __forceinline__ bool is_log_kernel(int kind)
{
    return kind == GSM_POISSON_2D || kind == GSM_DAVEY_STEWARTSON_2D;
}
__host__ __device__ __forceinline__ bool is_power_kernel(int kind)
{
    return kind == GSM_POWER_3D || kind == GSM_POWER_2D;
}

// What the Gaussian-sum kernels need to know about the sum being built.
struct GsSpec {
    int kind;                   // kernel whose sum is built
    double delta, rmax;         // interval [delta, rmax] of the error
    double beta;                // power kernels: exponent,
    double s_lo, s_hi;          //   node range in s,
    double cgam;                //   2 / Gamma(beta / 2)
};

// ---------------------------------------------------------------- Sec. 3: GS terms
// Coulomb (Sec. 3.2): 1/r = (1/sqrt(pi)) int_R exp(-r^2 sinh^2 t) cosh t dt,
// sinc nodes t = q theta, theta = 2.1 ln S / S; the even integrand folds the
// nodes +-q theta into one term.  nt = S + 1.
__device__ void coulomb_term(int q, int S, double &w, double &tau)
{
    const double th = 2.1 * log((double)S) / (double)S;
    if (q == 0) {
        w = th / kSqrtPi;
        tau = 0.0;
    } else {
        const double t = q * th;
        w = 2.0 * th * cosh(t) / kSqrtPi;
        tau = sinh(t);
    }
}

// ln r (Sec. 3.3), after the scaling of the 1/r^2 sum from [1, R] to
// [delta, rmax]: ln r = ln delta + 1/2 int_0^inf (e^-t - e^{-(r/delta)^2 t}) dt/t,
// t = ln(1 + exp(sinh s)), sinc nodes s = k theta, theta = ln S / S, k = -S..S.
// Node q = k + S + 1 (q = 1..2S+1) carries w = -theta t'(s)/(2 t(s)) and
// tau = sqrt(t)/delta; the constant term q = 0 is ln(delta) + sum theta t'/(2t) e^-t.
__device__ void log_node(int k, int S, double &t, double &tp_over_t)
{
    const double th = log((double)S) / (double)S;
    const double s = k * th;
    const double x = sinh(s);
    if (x < -36.0) {            // exp(x) < 3e-16: t = exp(x) to double precision
        t = exp(x);
        tp_over_t = cosh(s);
    } else if (x > 36.0) {      // t = x + log1p(exp(-x)), dt/dx = 1 to double precision
        t = x + log1p(exp(-x));
        tp_over_t = cosh(s) / t;
    } else {
        t = log1p(exp(x));
        tp_over_t = cosh(s) / ((1.0 + exp(-x)) * t);
    }
}

// r^-beta (remark after Eq. sinc_quad): Eq. Gauss_int with alpha = beta - 1,
// r^-beta = (2/Gamma(beta/2)) int_0^inf tau^(beta-1) exp(-r^2 tau^2) dtau, and
// with tau = exp(s - e^-s) (double-exponential decay at both ends of the s
// axis) the integrand in s is (2/Gamma(beta/2)) tau^beta (1 + e^-s) exp(-r^2 tau^2).
// S+1 sinc nodes with step (s_hi - s_lo)/S.
__device__ void power_term(int q, int S, const GsSpec &g, double &w, double &tau)
{
    const double h = (g.s_hi - g.s_lo) / (double)S;
    const double s = g.s_lo + q * h;
    const double em = exp(-s);
    const double ln_tau = s - em;
    tau = exp(ln_tau);
    w = g.cgam * h * (1.0 + em) * exp(g.beta * ln_tau);
}

// Block-cooperative construction of all terms into w[], tau[] (shared or
// global).  Returns nt.  Uses red[] (blockDim.x doubles of shared memory) for
// the constant C0 of the log kernel.
__device__ int build_terms(const GsSpec &gs, int S, double *w, double *tau, double *red)
{
    const int kind = gs.kind;
    const double delta = gs.delta;
    if (is_power_kernel(kind)) {
        const int nt = S + 1;
        for (int q = threadIdx.x; q < nt; q += blockDim.x) power_term(q, S, gs, w[q], tau[q]);
        __syncthreads();
        return nt;
    }
    if (!is_log_kernel(kind)) {
        const int nt = S + 1;
        for (int q = threadIdx.x; q < nt; q += blockDim.x) coulomb_term(q, S, w[q], tau[q]);
        __syncthreads();
        return nt;
    }
    const int nt = 2 * S + 2;
    const double th = log((double)S) / (double)S;
    double part = 0.0;
    for (int q = 1 + threadIdx.x; q < nt; q += blockDim.x) {
        double t, tpt;
        log_node(q - 1 - S, S, t, tpt);
        const double wt = 0.5 * th * tpt;
        part += wt * exp(-t);
        w[q] = -wt;
        tau[q] = sqrt(t) / delta;
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        w[0] = log(delta) + red[0];
        tau[0] = 0.0;
    }
    __syncthreads();
    return nt;
}

// One block per candidate S: maximum error over the sample.
__global__ void k_gs_scan(GsSpec gs, int S0, double *err_out)
{
    __shared__ double w[kGsCap], tau[kGsCap], red[1024];
    const int S = S0 + blockIdx.x;
    const int nt = build_terms(gs, S, w, tau, red);
    const int kind = gs.kind;
    const double delta = gs.delta, rmax = gs.rmax;
    double emax = 0.0;
    for (int i = threadIdx.x; i < kNSample + 2; i += blockDim.x) {
        double r;
        if (i == kNSample) r = delta;
        else if (i == kNSample + 1) r = rmax;
        else r = delta * pow(rmax / delta, (i + 0.5) / kNSample);
        double g = 0.0;
        for (int q = 0; q < nt; ++q) {
            const double a = tau[q] * r;
            g += w[q] * exp(-a * a);
        }
        double e;
        if (is_log_kernel(kind)) e = fabs(log(r) - g);
        else if (is_power_kernel(kind)) e = fabs(1.0 - pow(r, gs.beta) * g);
        else e = fabs(1.0 - r * g);
        emax = fmax(emax, e);
    }
    __syncthreads();
    red[threadIdx.x] = emax;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x == 0) err_out[blockIdx.x] = red[0];
}

__global__ void k_gs_terms(GsSpec gs, int S, double *w, double *tau)
{
    __shared__ double red[1024];
    build_terms(gs, S, w, tau, red);
}

// Node range of the r^-beta sum.  Left end: the part of the integral below
// tau_lo is at most (2/Gamma(beta/2)) tau_lo^beta / beta; it is set to eps/4
// times rmax^-beta, the smallest kernel value.  Right end: relative to r^-beta
// the part above tau_hi is the regularised upper incomplete gamma
// Q(beta/2, r^2 tau_hi^2), largest at r = delta; delta^2 tau_hi^2 = ln(1/eps) + 10
// puts it below eps/4 for beta < 3.  Each end is the root of
// f(s) = s - e^-s - ln tau, found by Newton steps from a point where f < 0:
// f is increasing and concave, so the steps climb to the root.
double s_of_ln_tau(double y)
{
    double s = (y < -1.0) ? -log(-y) : y - 1.0;
    for (int i = 0; i < 200; ++i) {
        const double em = exp(-s);
        const double step = (s - em - y) / (1.0 + em);
        s -= step;
        if (!(fabs(step) > 1e-15 * (1.0 + fabs(s)))) break;
    }
    return s;
}

void power_node_range(double beta, double delta, double rmax, double eps, double *s_lo, double *s_hi,
                      double *cgam)
{
    *cgam = 2.0 / std::tgamma(0.5 * beta);
    const double ln_tau_lo = (log(0.25 * eps * beta / *cgam) - beta * log(rmax)) / beta;
    const double ln_tau_hi = 0.5 * log(log(1.0 / eps) + 10.0) - log(delta);
    *s_lo = s_of_ln_tau(ln_tau_lo);
    *s_hi = s_of_ln_tau(ln_tau_hi);
}

// ---------------------------------------------------------------- Faddeeva w(z)
// Rational approximation of J. A. C. Weideman, "Computation of the complex
// error function", SIAM J. Numer. Anal. 31 (1994): with L = 2^(-1/4) sqrt(N),
// Z = (L + iz)/(L - iz),
//   w(z) ~ 2 sum_{n<N} a_{n+1} Z^n / (L - iz)^2 + 1 / (sqrt(pi) (L - iz)),
// a_j = (1/2M) sum_{|k|<M} f(t_k) cos(j theta_k), M = 2N, theta_k = k pi/M,
// t_k = L tan(theta_k/2), f(t) = exp(-t^2) (L^2 + t^2).  Valid for Im z >= 0.
__global__ void k_weideman(double *a)
{
    const int j = threadIdx.x + 1;
    if (j > kWeidN) return;
    const int M = 2 * kWeidN;
    const double L = sqrt(kWeidN / sqrt(2.0));
    double s = 0.0;
    for (int k = -M + 1; k < M; ++k) {
        const double th = k * kPi / M;
        const double t = L * tan(0.5 * th);
        s += exp(-t * t) * (L * L + t * t) * cos(j * th);
    }
    a[j - 1] = s / (2.0 * M);
}

struct zc {
    double re, im;
};
__device__ __forceinline__ zc zmul(zc a, zc b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ zc zdiv(zc a, zc b)
{
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

__device__ zc faddeeva(zc z, const double *a)
{
    const double L = sqrt(kWeidN / sqrt(2.0));
    const zc iz = {-z.im, z.re};
    const zc lm = {L - iz.re, -iz.im};      // L - iz
    const zc lp = {L + iz.re, iz.im};       // L + iz
    const zc Z = zdiv(lp, lm);
    zc p = {a[kWeidN - 1], 0.0};
    for (int nn = kWeidN - 2; nn >= 0; --nn) {
        p = zmul(p, Z);
        p.re += a[nn];
    }
    const zc lm2 = zmul(lm, lm);
    zc r = zdiv({2.0 * p.re, 2.0 * p.im}, lm2);
    const zc t = zdiv({1.0 / kSqrtPi, 0.0}, lm);
    return {r.re + t.re, r.im + t.im};
}

// ---------------------------------------------------------------- Eq. tensor factors
// g(tau, k) = int_{-2}^{2} exp(-tau^2 y^2) cos(omega y) dy, omega = pi k / 2
// (period 4 of the zero-padded box).  Three exact representations:
//  tau >= 4      : sqrt(pi)/tau exp(-omega^2/4tau^2); the part of the Gaussian
//                  beyond |y| = 2 is below exp(-64).
//  1 <= tau < 4  : completing the square,
//                  g = sqrt(pi)/tau [exp(-omega^2/4tau^2) - (-1)^k exp(-4tau^2) Re w(z)],
//                  z = -omega/(2 tau) + 2 i tau, w the Faddeeva function.
//  tau < 1       : series in tau^2, g = 2 sum_j (-4 tau^2)^j / j! m_j(pi k),
//                  m_j(nu) = int_{-1}^{1} x^{2j} cos(nu x) dx by the two-term
//                  recurrence m_j = (4j (-1)^k - 2j(2j-1) m_{j-1}) / nu^2 (from two
//                  integrations by parts; sin(nu) = 0), run upward while it is
//                  stable (2j(2j-1) < nu^2) and downward from far above otherwise.
__device__ double factor_g(double tau, int k, const double *weid)
{
    const double om = 0.5 * kPi * k;
    if (tau == 0.0) return k == 0 ? 4.0 : 0.0;
    if (tau >= kTauGauss) return kSqrtPi / tau * exp(-om * om / (4.0 * tau * tau));
    const double sgn = (k & 1) ? -1.0 : 1.0;
    if (tau >= kTauSeries) {
        const zc w = faddeeva({-om / (2.0 * tau), 2.0 * tau}, weid);
        return kSqrtPi / tau * (exp(-om * om / (4.0 * tau * tau)) - sgn * exp(-4.0 * tau * tau) * w.re);
    }
    double m[kTaylorJ];
    if (k == 0) {
        for (int j = 0; j < kTaylorJ; ++j) m[j] = 2.0 / (2 * j + 1);
    } else {
        const double nu = kPi * k, nu2 = nu * nu;
        m[0] = 0.0;
        int j = 1;
        for (; j < kTaylorJ && 2.0 * j * (2.0 * j - 1.0) < nu2; ++j)
            m[j] = (4.0 * j * sgn - 2.0 * j * (2.0 * j - 1.0) * m[j - 1]) / nu2;
        if (j < kTaylorJ) {
            // downward from jb; the start value's error shrinks by nu^2/(2j(2j-1))
            // (< 1/4 above 2 nu) per step
            const int jb = (int)fmax((double)kTaylorJ, 2.0 * nu) + 48;
            double mm = 2.0 * sgn / (2 * jb + 1);
            for (int jj = jb; jj > j; --jj) {
                mm = (4.0 * jj * sgn - nu2 * mm) / (2.0 * jj * (2.0 * jj - 1.0));
                if (jj - 1 < kTaylorJ) m[jj - 1] = mm;
            }
        }
    }
    const double x = -4.0 * tau * tau;
    double term = 1.0, s = 0.0;
    for (int j = 0; j < kTaylorJ; ++j) {
        s += term * m[j];
        term *= x / (j + 1);
    }
    return 2.0 * s;
}

// Axis of half-width eta (Sec. 2.5, Eq. tensor_ani): kernel box [-2 eta, 2 eta],
// period 4 eta; substituting y = eta y' gives eta * g(tau eta, k).
__global__ void k_factors(int nt, const double *tau, int nk, double eta, const double *weid, double *g)
{
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)nt * nk) return;
    const int q = idx / nk, k = idx - (long)q * nk;
    g[idx] = eta * factor_g(tau[q] * eta, k, weid);
}

// ---------------------------------------------------------------- Sec. 2.3 coefficients
// mu_m(tau) = int_0^delta r^m exp(-tau^2 r^2) dr: power series in x = tau delta
// for x <= 2, incomplete-gamma closed forms (m = 1..4) above.
__device__ double gauss_moment(int m, double tau, double delta)
{
    const double x = tau * delta;
    if (x <= 2.0) {
        const double x2 = x * x;
        double term = 1.0, s = 0.0;
        for (int j = 0; j < 80; ++j) {
            s += term / (m + 1 + 2 * j);
            term *= -x2 / (j + 1);
            if (fabs(term) < 1e-22) break;
        }
        return pow(delta, m + 1) * s;
    }
    const double e = exp(-x * x);
    const double t2 = tau * tau;
    switch (m) {
    case 1: return -expm1(-x * x) / (2.0 * t2);
    case 2: return kSqrtPi / (4.0 * t2 * tau) * erf(x) - delta * e / (2.0 * t2);
    case 3: return (1.0 - e * (1.0 + x * x)) / (2.0 * t2 * t2);
    default: return 3.0 * kSqrtPi / (8.0 * t2 * t2 * tau) * erf(x) -
                    e * (delta * delta * delta / (2.0 * t2) + 3.0 * delta / (4.0 * t2 * t2));
    }
}

// c0 = |S^{d-1}| A_{d-1}, c2 = |S^{d-1}|/(2d) A_{d+1},
// A_m = int_0^delta r^m (U1(r) - U_GS(r)) dr, U1 = 1/r, ln r or r^-beta.
__global__ void k_taylor(int kind, double beta, int d, int nt, const double *w, const double *tau, double delta,
                         double *out)
{
    __shared__ double r0[256], r1[256];
    double s0 = 0.0, s1 = 0.0;
    for (int q = threadIdx.x; q < nt; q += blockDim.x) {
        s0 += w[q] * gauss_moment(d - 1, tau[q], delta);
        s1 += w[q] * gauss_moment(d + 1, tau[q], delta);
    }
    r0[threadIdx.x] = s0;
    r1[threadIdx.x] = s1;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            r0[threadIdx.x] += r0[threadIdx.x + off];
            r1[threadIdx.x] += r1[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double area = d == 3 ? 4.0 * kPi : 2.0 * kPi;
        double e0, e1;
        const int m0 = d - 1, m1 = d + 1;
        if (is_log_kernel(kind)) {
            const double ld = log(delta);
            e0 = pow(delta, m0 + 1) * (ld / (m0 + 1) - 1.0 / ((m0 + 1.0) * (m0 + 1.0)));
            e1 = pow(delta, m1 + 1) * (ld / (m1 + 1) - 1.0 / ((m1 + 1.0) * (m1 + 1.0)));
        } else if (is_power_kernel(kind)) {
            e0 = pow(delta, m0 + 1 - beta) / (m0 + 1 - beta);   // beta < d = m0 + 1
            e1 = pow(delta, m1 + 1 - beta) / (m1 + 1 - beta);
        } else {
            e0 = pow(delta, m0) / m0;
            e1 = pow(delta, m1) / m1;
        }
        out[0] = area * (e0 - r0[0]);
        out[1] = area / (2.0 * d) * (e1 - r1[0]);
    }
}

// ---------------------------------------------------------------- tensor and multiplier
// khat[kx][ky][kz] = sum_q w_q g0[q][kx] g1[q][ky] g2[q][kz]  (kz fastest)
__global__ void k_tensor(int d, int n0, int n1, int n2, int nt, const double *w, const double *g0,
                         const double *g1, const double *g2, double *khat)
{
    const long tot = (long)(n0 + 1) * (n1 + 1) * (d == 3 ? n2 + 1 : 1);
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int h1 = n1 + 1, h2 = d == 3 ? n2 + 1 : 1;
    const int kz = d == 3 ? idx % h2 : 0;
    const int ky = d == 3 ? (idx / h2) % h1 : idx % h1;
    const int kx = d == 3 ? idx / ((long)h1 * h2) : idx / h1;
    double s = 0.0;
    for (int q = 0; q < nt; ++q) {
        double t = w[q] * g0[(long)q * (n0 + 1) + kx] * g1[(long)q * (n1 + 1) + ky];
        if (d == 3) t *= g2[(long)q * (n2 + 1) + kz];
        s += t;
    }
    khat[idx] = s;
}

struct MultParams {
    int d, kind, n[3], M[3];
    double eta[3];      // axis half-widths in units of L (Sec. 2.5)
    double scale;       // s of Sec. 2.1
    double c0, c2;
    double norm;        // 1/2 (pair packing of the real x transform) / prod M
    double extra0;      // Poisson: -(L^2/2pi) ln L * P^d at k = 0
    int dip_axis;       // >= 0: dipolar with n, m along this axis
    double dip_nm;      // n.m
    double L;
};

// multiplier = norm * ( scale (khat + c0 - c2 |kappa|^2) [+ extra0 at k=0] ),
// dipolar along axis a: norm * ( -(n.m) + 3 (n.m) kappa_a^2 / L^2 * scale (...) ).
// kappa_j = pi k_j / 2 in unit-box coordinates (period 4).
__global__ void k_multiplier(MultParams mp, const double *khat, double *mult)
{
    const int d = mp.d;
    const int h1 = mp.n[1] + 1, h2 = d == 3 ? mp.n[2] + 1 : 1;
    const long tot = (long)(mp.n[0] + 1) * h1 * h2;
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int kz = d == 3 ? idx % h2 : 0;
    const int ky = d == 3 ? (idx / h2) % h1 : idx % h1;
    const int kx = d == 3 ? idx / ((long)h1 * h2) : idx / h1;
    const int k[3] = {kx, ky, kz};
    double kap2 = 0.0;
    for (int j = 0; j < d; ++j) {
        const double kap = 0.5 * kPi * k[j] / mp.eta[j];   // 2 pi k / (4 eta_j)
        kap2 += kap * kap;
    }
    double v = mp.scale * (khat[idx] + mp.c0 - mp.c2 * kap2);
    if (mp.kind == GSM_POISSON_2D && idx == 0) v += mp.extra0;
    if (mp.kind == GSM_DAVEY_STEWARTSON_2D) {
        // source d_xx rho: symbol -kappa_x^2 in physical units; its k = 0 mode
        // vanishes, and with it the ln L term of the rescaling
        const double kx = 0.5 * kPi * k[0] / mp.eta[0];
        v *= -kx * kx / (mp.L * mp.L);
    }
    if (mp.kind == GSM_DIPOLAR_3D) {
        const double ka = 0.5 * kPi * k[mp.dip_axis] / mp.eta[mp.dip_axis];
        v = -mp.dip_nm + 3.0 * mp.dip_nm * ka * ka / (mp.L * mp.L) * v;
    }
    mult[idx] = v * mp.norm;
}


// General dipolar directions (Sec. 2.4, Example 4): the multiplier
//   norm (-(n.m)) + 3 (n.kappa')(m.kappa')' / L^2 * mC(|k|),
// mC the normalised Coulomb multiplier on the octant.  (n.k)(m.k) is even under
// k -> -k but not per axis, so it is stored for every (kx >= 0, ky, kz) of the
// half spectrum, row (kx * My + ky) of Mz entries.  First derivatives vanish at
// the Nyquist index: sum_ij n_i m_j k_i k_j drops the terms i != j in which
// k_i or k_j is the Nyquist frequency.
struct DipFull {
    int n[3], M[3];
    double eta[3];
    double nv[3], mv[3];
    double L, norm;
    int prec;
};

__global__ void k_multiplier_dip_full(DipFull dp, const double *__restrict__ mC, void *out)
{
    const int hx = dp.n[0] + 1, My = dp.M[1], Mz = dp.M[2];
    const long tot = (long)hx * My * Mz;
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int kz = idx % Mz, ky = (idx / Mz) % My, kx = idx / ((long)Mz * My);
    const int kk[3] = {kx, ky < My - ky ? ky : ky - My, kz < Mz - kz ? kz : kz - Mz};
    double kap[3];
    bool nyq[3];
    for (int j = 0; j < 3; ++j) {
        kap[j] = 0.5 * kPi * kk[j] / dp.eta[j];
        nyq[j] = 2 * (kk[j] < 0 ? -kk[j] : kk[j]) == dp.M[j];
    }
    double sym = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (i != j && (nyq[i] || nyq[j])) continue;
            sym += dp.nv[i] * dp.mv[j] * kap[i] * kap[j];
        }
    const int fy = ky < My - ky ? ky : My - ky, fz = kz < Mz - kz ? kz : Mz - kz;
    const double c = mC[((size_t)kx * (dp.n[1] + 1) + fy) * (dp.n[2] + 1) + fz];
    const double nm = dp.nv[0] * dp.mv[0] + dp.nv[1] * dp.mv[1] + dp.nv[2] * dp.mv[2];
    const double v = -nm * dp.norm + 3.0 * sym / (dp.L * dp.L) * c;
    if (dp.prec == GSM_FP64) {
        reinterpret_cast<double *>(out)[idx] = v;
    } else if (dp.prec == GSM_FP32) {
        reinterpret_cast<float *>(out)[idx] = (float)v;
    } else {
        const df a = df_from_double(v);
        reinterpret_cast<float2 *>(out)[idx] = make_float2(a.hi, a.lo);
    }
}
}  // namespace

// ---------------------------------------------------------------- host side
// Results of the Gaussian-sum scan (the chosen S and its error), kept for the
// process: plans of other grid sizes with the same kernel, delta, interval,
// accuracy target (and beta) reuse them.  The scan is deterministic, so a hit
// gives what the scan would.
namespace {
struct GsKey {
    int device, kind, S_request;
    double delta, rmax, eps, beta;
    bool operator<(const GsKey &o) const
    {
        return std::tie(device, kind, S_request, delta, rmax, eps, beta) <
               std::tie(o.device, o.kind, o.S_request, o.delta, o.rmax, o.eps, o.beta);
    }
};
std::mutex g_gs_mutex;
std::map<GsKey, std::pair<int, double>> g_gs_cache;

GsKey gs_key(const GsSpec &gs, int S_request, double eps)
{
    int dev = 0;
    cudaGetDevice(&dev);
    return GsKey{dev, gs.kind, S_request, gs.delta, gs.rmax, eps, gs.beta};
}

bool gs_cache_lookup(const GsSpec &gs, int S_request, double eps, int *S, double *err)
{
    std::lock_guard<std::mutex> lock(g_gs_mutex);
    auto it = g_gs_cache.find(gs_key(gs, S_request, eps));
    if (it == g_gs_cache.end()) return false;
    *S = it->second.first;
    *err = it->second.second;
    return true;
}

void gs_cache_insert(const GsSpec &gs, int S_request, double eps, int S, double err)
{
    std::lock_guard<std::mutex> lock(g_gs_mutex);
    g_gs_cache[gs_key(gs, S_request, eps)] = {S, err};
}
}  // namespace

gsm_status_t build_plan_data(Plan *p, cudaStream_t st, const StoredPlanData *stored)
{
    const int d = p->d;
    const double delta = p->opt.delta;
    // the kernel box has half-widths 2 eta_a: its corners lie at 2 |eta|
    double eta2 = 0.0;
    for (int a = 0; a < d; ++a) eta2 += p->eta[a] * p->eta[a];
    const double rmax = 2.0 * sqrt(eta2);
    // the dipolar potential is built on the Coulomb sum, Davey-Stewartson on ln r
    const int kind_gs = p->kind == GSM_DIPOLAR_3D ? GSM_COULOMB_3D
                        : (p->kind == GSM_DAVEY_STEWARTSON_2D ? GSM_POISSON_2D : p->kind);

    GSM_CUDA_TRY(dev_alloc(&p->d_w, sizeof(double) * kGsCap));
    GSM_CUDA_TRY(dev_alloc(&p->d_tau, sizeof(double) * kGsCap));
    GsSpec gs;
    gs.kind = kind_gs;
    gs.delta = delta;
    gs.rmax = rmax;
    gs.beta = p->opt.beta;
    gs.s_lo = gs.s_hi = 0.0;
    gs.cgam = 0.0;
    if (is_power_kernel(kind_gs)) power_node_range(gs.beta, delta, rmax, p->eps, &gs.s_lo, &gs.s_hi, &gs.cgam);

    // 1. choose S (smallest meeting eps), scanning a first window then the rest
    int S = stored ? stored->S : p->opt.S;
    double err = stored ? stored->gs_err : 0.0;
    if (S > kSmax || S < 0) {
        set_error("options.S must be in [0, 500]");
        return GSM_ERR_INVALID_ARG;
    }
    if (stored) {
        const int want = (kind_gs == GSM_POISSON_2D) ? 2 * S + 2 : S + 1;
        if (S < 1 || stored->nterms != want || stored->nterms > kGsCap) {
            set_error("stored plan: Gaussian-sum size does not match its kernel");
            return GSM_ERR_INVALID_ARG;
        }
    } else if (gs_cache_lookup(gs, p->opt.S, p->eps, &S, &err)) {
        // the same scan ran for an earlier plan in this process
    } else {
        const int S_request = S;
        DevTemp err_buf;
        const int S_first = 4;
        const int count = kSmax - S_first + 1;
        GSM_CUDA_TRY(dev_alloc(&err_buf.p, sizeof(double) * count));
        double *d_err = err_buf.as<double>();
        std::vector<double> h(count, INFINITY);
        const int windows[3][2] = {{S_first, 160}, {161, 320}, {321, kSmax}};
        bool found = false;
        for (int wi = 0; wi < 3 && !found; ++wi) {
            int a = windows[wi][0], b = windows[wi][1];
            if (S > 0) {
                if (S < a || S > b) continue;
                a = b = S;
            }
            k_gs_scan<<<b - a + 1, 256, 0, st>>>(gs, a, d_err + (a - S_first));
            cudaError_t e = cudaMemcpyAsync(h.data() + (a - S_first), d_err + (a - S_first),
                                            sizeof(double) * (b - a + 1), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                set_error(std::string("Gaussian-sum scan: ") + cudaGetErrorString(e));
                return GSM_ERR_CUDA;
            }
            for (int s = a; s <= b; ++s) {
                if (S > 0 || h[s - S_first] <= p->eps) {
                    S = s;
                    err = h[s - S_first];
                    found = true;
                    break;
                }
            }
        }
        if (!found) {
            set_error("no Gaussian sum with S <= 500 meets the requested accuracy");
            return GSM_ERR_ACCURACY;
        }
        gs_cache_insert(gs, S_request, p->eps, S, err);
    }
    p->S = S;
    p->gs_err = err;
    p->nterms = (kind_gs == GSM_POISSON_2D) ? 2 * S + 2 : S + 1;
    if (stored) {
        GSM_CUDA_TRY(cudaMemcpyAsync(p->d_w, stored->w, sizeof(double) * p->nterms, cudaMemcpyHostToDevice, st));
        GSM_CUDA_TRY(cudaMemcpyAsync(p->d_tau, stored->tau, sizeof(double) * p->nterms, cudaMemcpyHostToDevice, st));
    } else {
        k_gs_terms<<<1, 1024, 0, st>>>(gs, S, p->d_w, p->d_tau);
    }

    // 2. 1-D factors per axis
    DevTemp weid_buf;
    GSM_CUDA_TRY(dev_alloc(&weid_buf.p, sizeof(double) * kWeidN));
    const double *d_weid = weid_buf.as<double>();
    k_weideman<<<1, kWeidN, 0, st>>>(weid_buf.as<double>());
    for (int a = 0; a < d; ++a) {
        const int nk = p->n[a] + 1;
        bool same = false;
        for (int b = 0; b < a; ++b)
            if (p->n[b] == p->n[a] && p->eta[b] == p->eta[a]) {
                p->d_g[a] = p->d_g[b];
                same = true;
                break;
            }
        if (same) continue;
        GSM_CUDA_TRY(dev_alloc(&p->d_g[a], sizeof(double) * p->nterms * nk));
        const long tot = (long)p->nterms * nk;
        k_factors<<<(tot + 127) / 128, 128, 0, st>>>(p->nterms, p->d_tau, nk, p->eta[a], d_weid, p->d_g[a]);
    }

    // 3. Taylor coefficients
    if (stored) {
        GSM_CUDA_TRY(cudaStreamSynchronize(st));
        p->c0 = stored->c0;
        p->c2 = stored->c2;
    } else {
        DevTemp c_buf;
        GSM_CUDA_TRY(dev_alloc(&c_buf.p, sizeof(double) * 2));
        k_taylor<<<1, 256, 0, st>>>(kind_gs, p->opt.beta, d, p->nterms, p->d_w, p->d_tau, delta,
                                    c_buf.as<double>());
        double hc[2];
        GSM_CUDA_TRY(cudaMemcpyAsync(hc, c_buf.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
        GSM_CUDA_TRY(cudaStreamSynchronize(st));
        p->c0 = hc[0];
        p->c2 = hc[1];
    }

    // 4. tensor and multiplier on the octant
    size_t tot = 1;
    for (int a = 0; a < d; ++a) tot *= (size_t)(p->n[a] + 1);
    p->mult_elems = tot;
    GSM_CUDA_TRY(dev_alloc(&p->d_khat, sizeof(double) * tot));
    GSM_CUDA_TRY(dev_alloc(&p->d_mult64, sizeof(double) * tot));
    if (stored)
        GSM_CUDA_TRY(cudaMemcpyAsync(p->d_khat, stored->khat, sizeof(double) * tot, cudaMemcpyHostToDevice, st));
    else
        k_tensor<<<(tot + 127) / 128, 128, 0, st>>>(d, p->n[0], p->n[1], p->n[2], p->nterms, p->d_w,
                                                      p->d_g[0], p->d_g[1], d > 2 ? p->d_g[2] : p->d_g[1],
                                                      p->d_khat);
    MultParams mp;
    mp.d = d;
    // general dipolar directions: the octant holds the Coulomb multiplier and
    // the dipolar symbol is applied in the full table built below
    mp.kind = (p->kind == GSM_DIPOLAR_3D && p->dip_axis < 0) ? GSM_COULOMB_3D : p->kind;
    for (int a = 0; a < 3; ++a) {
        mp.n[a] = p->n[a];
        mp.M[a] = p->M[a];
        mp.eta[a] = p->eta[a];
    }
    const double L = p->L;
    if (p->kind == GSM_COULOMB_3D || p->kind == GSM_DIPOLAR_3D) mp.scale = L * L / (4.0 * kPi);
    else if (p->kind == GSM_COULOMB_2D) mp.scale = L / (2.0 * kPi);
    else if (is_power_kernel(p->kind)) mp.scale = pow(L, d - p->opt.beta);   // |L x|^-beta L^d
    else mp.scale = -L * L / (2.0 * kPi);   // ln kernel: Poisson and Davey-Stewartson
    mp.c0 = p->c0;
    mp.c2 = p->c2;
    double pm = 1.0;
    for (int a = 0; a < d; ++a) pm *= p->M[a];
    mp.norm = 0.5 / pm;
    // Poisson: -(L^2/2pi) ln L int rho~, and int rho~ = prod h_a sum rho with
    // h_a M_a = 4 eta_a, so the k = 0 entry gains the constant times prod 4 eta_a
    double vol = 1.0;
    for (int a = 0; a < d; ++a) vol *= 4.0 * p->eta[a];
    mp.extra0 = (p->kind == GSM_POISSON_2D) ? -L * L / (2.0 * kPi) * log(L) * vol : 0.0;
    mp.dip_axis = p->dip_axis;
    mp.dip_nm = p->opt.dip_n[0] * p->opt.dip_m[0] + p->opt.dip_n[1] * p->opt.dip_m[1] +
                p->opt.dip_n[2] * p->opt.dip_m[2];
    mp.L = L;
    k_multiplier<<<(tot + 127) / 128, 128, 0, st>>>(mp, p->d_khat, p->d_mult64);
    GSM_CUDA_TRY(cudaGetLastError());

    // twiddles and the pass-precision multiplier
    for (int a = 0; a < d; ++a) {
        gsm_status_t s = make_twiddles(p, a, st);
        if (s != GSM_OK) return s;
    }
    if (p->split_conv) {
        gsm_status_t s = make_split_tables(p, st);
        if (s != GSM_OK) return s;
    }
    if (p->split_x) {
        gsm_status_t s = make_xsplit_tables(p, st);
        if (s != GSM_OK) return s;
    }
    if (p->kind == GSM_DIPOLAR_3D && p->dip_axis < 0) {
        DipFull dp;
        for (int a = 0; a < 3; ++a) {
            dp.n[a] = p->n[a];
            dp.M[a] = p->M[a];
            dp.eta[a] = p->eta[a];
            dp.nv[a] = p->opt.dip_n[a];
            dp.mv[a] = p->opt.dip_m[a];
        }
        dp.L = L;
        dp.norm = mp.norm;
        dp.prec = p->opt.precision;
        const size_t full = (size_t)(p->n[0] + 1) * p->M[1] * p->M[2];
        const size_t eb = p->opt.precision == GSM_FP32 ? sizeof(float) : sizeof(double);
        GSM_CUDA_TRY(dev_alloc(&p->d_mult, eb * full));
        p->mult_full = true;
        p->mult_elems_pass = full;
        k_multiplier_dip_full<<<(full + 255) / 256, 256, 0, st>>>(dp, p->d_mult64, p->d_mult);
        GSM_CUDA_TRY(cudaGetLastError());
        GSM_CUDA_TRY(cudaStreamSynchronize(st));
        return GSM_OK;
    }
    p->mult_elems_pass = p->mult_elems;
    gsm_status_t s = make_pass_multiplier(p, st);
    if (s != GSM_OK) return s;
    GSM_CUDA_TRY(cudaStreamSynchronize(st));
    return GSM_OK;
}

}  // namespace gsm
