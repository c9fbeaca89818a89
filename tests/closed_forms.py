"""Closed-form potentials of Gaussian densities printed in Sec. 4 of the paper,
evaluated with scipy.special (an independent library).  Test infrastructure."""
import numpy as np
from scipy import integrate
from scipy.special import erf, exp1, i0e


def coulomb3d_gaussian(r, sigma):
    """Eq. DensGaus, gamma = 1: sigma^3 sqrt(pi) erf(r/sigma) / (4 r)."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    small = r < 1e-8 * sigma
    rr = np.where(small, 1.0, r)
    out[:] = sigma ** 3 * np.sqrt(np.pi) * erf(rr / sigma) / (4.0 * rr)
    out[small] = sigma ** 2 / 2.0
    return out


def coulomb3d_gaussian_axes(X, Y, Z, s):
    """Potential of exp(-(x/s0)^2 - (y/s1)^2 - (z/s2)^2) for U = 1/(4 pi |x|), from
    1/r = (2/sqrt(pi)) int_0^inf exp(-r^2 t^2) dt (Eq. GauInte) and the Gaussian
    integral per axis:  u = (1/(4pi)) (2/sqrt(pi)) int_0^inf prod_i sqrt(pi/(t^2 + s_i^-2))
    exp(-t^2 x_i^2 s_i^-2 / (t^2 + s_i^-2)) dt, evaluated pointwise by quadrature."""
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    a = 1.0 / np.asarray(s, dtype=np.float64) ** 2
    out = np.empty(len(pts))
    for i, x in enumerate(pts):
        def f(t):
            v = 1.0
            for j in range(3):
                v *= np.sqrt(np.pi / (t * t + a[j])) * np.exp(-t * t * a[j] * x[j] ** 2 / (t * t + a[j]))
            return v
        val, _ = integrate.quad(f, 0, np.inf, epsabs=0, epsrel=1e-13, limit=400)
        out[i] = val * 2.0 / np.sqrt(np.pi) / (4.0 * np.pi)
    return out.reshape(X.shape)


def coulomb2d_gaussian(r, sigma):
    """Eq. 2.5D-clb-exact, gamma = 1: (sqrt(pi) sigma/2) I0(r^2/2s^2) exp(-r^2/2s^2)."""
    return np.sqrt(np.pi) * sigma / 2.0 * i0e(np.asarray(r) ** 2 / (2.0 * sigma ** 2))


def poisson2d_gaussian(r, sigma):
    """Eq. eg-2d-Exact: -(s^2/4)[E1(r^2/s^2) + 2 ln r], origin (s^2/4)(gamma_e - ln s^2)."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    z = r == 0
    rr = np.where(z, 1.0, r)
    out[:] = -(sigma ** 2 / 4.0) * (exp1(rr ** 2 / sigma ** 2) + 2.0 * np.log(rr))
    out[z] = sigma ** 2 / 4.0 * (np.euler_gamma - np.log(sigma ** 2))
    return out


def dipolar3d_gaussian(X, Y, Z, sigma, nv, mv):
    """Example 4: u = -(n.m) rho - 3 n^T D m with the Hessian D printed there;
    at the origin D = -I/3 (its limit), so u(0) = 0 for rho(0) = 1."""
    nv = np.asarray(nv, dtype=np.float64)
    mv = np.asarray(mv, dtype=np.float64)
    r2 = X * X + Y * Y + Z * Z
    r = np.sqrt(r2)
    s = sigma
    e = np.exp(-r2 / s ** 2)
    z = r == 0
    rr = np.where(z, 1.0, r)
    r2s = rr * rr
    ef = erf(rr / s)
    a = s ** 2 / (2 * r2s) * e - s ** 3 * np.sqrt(np.pi) / (4 * rr ** 3) * ef
    b = -3 * s ** 2 / (2 * r2s ** 2) * e - e / r2s + 3 * s ** 3 * np.sqrt(np.pi) / (4 * rr ** 5) * ef
    xs = (X, Y, Z)
    nx = sum(nv[i] * xs[i] for i in range(3))
    mx = sum(mv[i] * xs[i] for i in range(3))
    u = -np.dot(nv, mv) * e - 3.0 * (a * np.dot(nv, mv) + b * nx * mx)
    u = np.where(z, -np.dot(nv, mv) * 1.0 + np.dot(nv, mv), u)
    return u


def ds2d_gaussian(X, Y):
    """Example 5: for rho = pi exp(-pi^2 r^2), u = -(1/2pi) ln|x| * d_xx rho is
    Phi = -( (pi/2) e^{-pi^2 r^2} + cos(2 theta) e^{-pi^2 r^2} (1 + pi^2 r^2 - e^{pi^2 r^2}) / (2 pi r^2) ),
    the second term written as (e^{-a}(1 + a) - 1)/(2 pi r^2), a = pi^2 r^2,
    which tends to 0 at the origin."""
    r2 = X * X + Y * Y
    a = np.pi ** 2 * r2
    th = np.arctan2(Y, X)
    z = r2 == 0
    rr = np.where(z, 1.0, r2)
    aa = np.where(z, 1.0, a)
    g = (np.exp(-aa) * (1.0 + aa) - 1.0) / (2.0 * np.pi * rr)
    g = np.where(z, 0.0, g)
    return -(np.pi / 2.0 * np.exp(-a) + np.cos(2.0 * th) * g)


def coulomb_gaussian_axes_points(points, widths, dim):
    """Coulomb potential (1/(4 pi |x|) in 3D, 1/(2 pi |x|) in 2D) of
    exp(-sum_i (x_i / s_i)^2) at the given points (shape (P, dim)), from
    1/r = (2/sqrt(pi)) int_0^inf exp(-r^2 t^2) dt (Eq. GauInte) and the Gaussian
    integral per axis, by adaptive quadrature in t."""
    a = 1.0 / np.asarray(widths, dtype=np.float64) ** 2
    pref = (1.0 / (4.0 * np.pi)) if dim == 3 else (1.0 / (2.0 * np.pi))
    out = np.empty(len(points))
    for k, x in enumerate(points):
        def f(t):
            v = 1.0
            for j in range(dim):
                v *= np.sqrt(np.pi / (t * t + a[j])) * np.exp(-t * t * a[j] * x[j] ** 2 / (t * t + a[j]))
            return v
        val, _ = integrate.quad(f, 0, np.inf, epsabs=0, epsrel=1e-13, limit=400)
        out[k] = pref * 2.0 / np.sqrt(np.pi) * val
    return out


def power_gaussian(r, sigma, beta, d):
    """Potential of exp(-|x|^2/sigma^2) under U = |x|^-beta in R^d (0 < beta < d):
    from r^-beta = (2/Gamma(beta/2)) int_0^inf tau^(beta-1) exp(-r^2 tau^2) dtau
    (Eq. Gauss_int, alpha = beta - 1) and the Gaussian convolution,
    u = pi^(d/2) sigma^(d-beta) Gamma((d-beta)/2)/Gamma(d/2) 1F1(beta/2; d/2; -r^2/sigma^2),
    the confluent hypergeometric function from scipy.special."""
    from scipy.special import gamma, hyp1f1
    r = np.asarray(r, dtype=np.float64)
    c = np.pi ** (d / 2) * sigma ** (d - beta) * gamma((d - beta) / 2) / gamma(d / 2)
    return c * hyp1f1(beta / 2, d / 2, -r * r / sigma ** 2)
