"""Plain FP64 CPU oracle for the Gaussian-sum method (Exl, Mauser, Zhang,
arXiv:1501.04438).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product (the
CUDA library in ``paper_1501_04438_gb300``) never imports it and shares no code
with it.  The arithmetic lives in ``oracle.c`` (plain C, double precision, each
quantity computed from the equation of the paper that defines it); this module
only builds that file and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KERNELS = {"coulomb3d": 0, "coulomb2d": 1, "poisson2d": 2, "dipolar3d": 3, "ds2d": 4, "power3d": 5, "power2d": 6}
KERNEL_DIM = {"coulomb3d": 3, "coulomb2d": 2, "poisson2d": 2, "dipolar3d": 3, "ds2d": 2, "power3d": 3,
              "power2d": 2}
GS_CAP = 1024

# Default accuracy targets of the Gaussian sums (Sec. 3.2-3.3): relative error
# of 1/r and absolute error of ln r over [delta, 2 sqrt(d)].  Both sit just above
# the rounding floor of the sums built in double (1/r: 0.9e-15 for delta = 1e-3,
# 1.2e-15 for delta = 1e-4; ln r: about 5e-14).
DEFAULT_EPS = {"coulomb3d": 2e-15, "coulomb2d": 2e-15, "dipolar3d": 2e-15, "poisson2d": 1e-13, "ds2d": 1e-13,
               "power3d": 2e-15, "power2d": 2e-15}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP if present)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_int),
        ("d", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("L", ctypes.c_double),
        ("pad", ctypes.c_int),
        ("delta", ctypes.c_double),
        ("gs_eps", ctypes.c_double),
        ("gs_S", ctypes.c_int),
        ("taylor_mode", ctypes.c_int),
        ("dip_n", ctypes.c_double * 3),
        ("dip_m", ctypes.c_double * 3),
        ("threads", ctypes.c_int),
        ("box", ctypes.c_double * 3),
        ("beta", ctypes.c_double),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("S", ctypes.c_int),
        ("nterms", ctypes.c_int),
        ("gs_err", ctypes.c_double),
        ("c0", ctypes.c_double),
        ("c2", ctypes.c_double),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.orc_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
            L.orc_gs_eval.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double]
            L.orc_gs_eval.restype = ctypes.c_double
            L.orc_gs_error.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int]
            L.orc_gs_error.restype = ctypes.c_double
            L.orc_gs_build.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _dp, _ip, _ip, _dp]
            L.orc_factor.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_factor.restype = ctypes.c_double
            L.orc_fftn.argtypes = [ctypes.c_int, _ip, _dp, ctypes.c_int]
            L.orc_taylor_coeffs.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                            ctypes.c_double, _dp, _dp]
            L.orc_kernel_hat.argtypes = [ctypes.POINTER(Params), _dp, ctypes.POINTER(Info)]
            L.orc_apply_parts.argtypes = [ctypes.POINTER(Params), _dp, _dp, _dp, _dp, ctypes.POINTER(Info)]
            L.orc_max_threads.restype = ctypes.c_int
            L.orc_prepare.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Info)]
            L.orc_prepare.restype = ctypes.c_void_p
            L.orc_run.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
            L.orc_free_prepared.argtypes = [ctypes.c_void_p]
            L.orc_free_prepared.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def gauss_legendre(m: int):
    x = np.zeros(m)
    w = np.zeros(m)
    lib().orc_gauss_legendre(m, _ptr(x), _ptr(w))
    return x, w


def gs(kernel: str, delta: float = 1e-3, eps: float | None = None, S: int = 0, rmax: float | None = None,
       beta: float = 1.0):
    """Gaussian sum (w_q, tau_q) of 1/r (Coulomb kernels), ln r (Poisson) or
    r^-beta (power kernels).

    Returns (w, tau, S, err), err being E_rel or E_abs on [delta, rmax]."""
    base = {"dipolar3d": "coulomb3d", "ds2d": "poisson2d"}.get(kernel, kernel)
    d = KERNEL_DIM[kernel]
    if rmax is None:
        rmax = 2.0 * np.sqrt(d)
    if eps is None:
        eps = DEFAULT_EPS[kernel]
    w = np.zeros(GS_CAP)
    tau = np.zeros(GS_CAP)
    nt = ctypes.c_int()
    So = ctypes.c_int()
    err = ctypes.c_double()
    rc = lib().orc_gs_build(KERNELS[base], float(beta), delta, rmax, eps, S, GS_CAP, _ptr(w), _ptr(tau),
                            ctypes.byref(nt), ctypes.byref(So), ctypes.byref(err))
    if rc != 0:
        raise RuntimeError("oracle: no Gaussian sum meets the requested accuracy")
    return w[: nt.value].copy(), tau[: nt.value].copy(), So.value, err.value


def gs_eval(w, tau, r):
    w = np.ascontiguousarray(w, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return np.array([lib().orc_gs_eval(len(w), _ptr(w), _ptr(tau), float(x)) for x in r])


def gs_error(kernel, w, tau, delta, rmax, ns=4000, beta: float = 1.0):
    base = {"dipolar3d": "coulomb3d", "ds2d": "poisson2d"}.get(kernel, kernel)
    w = np.ascontiguousarray(w, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    return lib().orc_gs_error(KERNELS[base], float(beta), len(w), _ptr(w), _ptr(tau), delta, rmax, ns)


def factor(tau: float, omega: float) -> float:
    """int_{-2}^{2} exp(-tau^2 y^2) cos(omega y) dy (one factor of Eq. tensor)."""
    return lib().orc_factor(float(tau), float(omega))


def fftn(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised DFT along every axis, exp(sign*2*pi*i*jk/n)."""
    c = np.ascontiguousarray(a, dtype=np.complex128).copy()
    shape = (ctypes.c_int * 3)(*(list(c.shape[::-1]) + [1] * (3 - c.ndim)))
    v = c.view(np.float64)
    lib().orc_fftn(c.ndim, shape, _ptr(v), sign)
    return c


def taylor_coeffs(kernel: str, w, tau, delta: float, beta: float = 1.0):
    base = {"dipolar3d": "coulomb3d", "ds2d": "poisson2d"}.get(kernel, kernel)
    d = KERNEL_DIM[kernel]
    w = np.ascontiguousarray(w, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    c0 = ctypes.c_double()
    c2 = ctypes.c_double()
    lib().orc_taylor_coeffs(KERNELS[base], float(beta), d, len(w), _ptr(w), _ptr(tau), delta,
                            ctypes.byref(c0), ctypes.byref(c2))
    return c0.value, c2.value


def make_params(kernel: str, n, L: float, pad: int = 2, delta: float = 1e-3, eps: float | None = None,
                S: int = 0, taylor_mode: int = 0, dip_n=(0.0, 0.0, 1.0), dip_m=(0.0, 0.0, 1.0),
                threads: int = 0, box=None, beta: float = 1.0) -> Params:
    """box: per-axis half-widths (x first) of a rectangular box; L is then unused.
    beta: exponent of the power kernels |x|^-beta."""
    d = KERNEL_DIM[kernel]
    if isinstance(n, int):
        n = [n] * d
    nn = list(n) + [1] * (3 - len(n))
    p = Params()
    p.kernel = KERNELS[kernel]
    p.d = d
    for i in range(3):
        p.n[i] = int(nn[i])
    p.L = float(L)
    p.pad = int(pad)
    p.delta = float(delta)
    p.gs_eps = float(DEFAULT_EPS[kernel] if eps is None else eps)
    p.gs_S = int(S)
    p.taylor_mode = int(taylor_mode)
    for i in range(3):
        p.dip_n[i] = float(dip_n[i])
        p.dip_m[i] = float(dip_m[i])
    p.threads = int(threads)
    bx = list(box) if box is not None else []
    for i in range(3):
        p.box[i] = float(bx[i]) if i < len(bx) else 0.0
    p.beta = float(beta)
    return p


def kernel_hat(kernel: str, n, L: float = 1.0, **kw):
    """Octant of sum_q w_q G_k^q, k_j = 0..pad*n_j/2, layout [kz][ky][kx]."""
    p = make_params(kernel, n, L, **kw)
    d = p.d
    no = [p.pad * p.n[a] // 2 + 1 for a in range(d)]
    out = np.zeros(int(np.prod(no)))
    info = Info()
    if lib().orc_kernel_hat(ctypes.byref(p), _ptr(out), ctypes.byref(info)) != 0:
        raise RuntimeError("oracle kernel_hat failed")
    return out.reshape(no[::-1]), info


def apply(kernel: str, rho: np.ndarray, L: float, parts: bool = False, **kw):
    """u = U * rho on the grid of Sec. 2.1 (x_i = -L + (i+1) h), Algorithm 1.

    rho is C-ordered with x fastest: shape (nz, ny, nx) or (ny, nx)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    p = make_params(kernel, list(rho.shape[::-1]), L, **kw)
    u = np.zeros_like(rho)
    i1 = np.zeros_like(rho) if parts else None
    i2 = np.zeros_like(rho) if parts else None
    info = Info()
    rc = lib().orc_apply_parts(ctypes.byref(p), _ptr(rho), _ptr(u), _ptr(i1), _ptr(i2), ctypes.byref(info))
    if rc != 0:
        raise RuntimeError("oracle apply failed (bad arguments or no Gaussian sum)")
    info_d = {"S": info.S, "nterms": info.nterms, "gs_err": info.gs_err, "c0": info.c0, "c2": info.c2}
    if parts:
        return u, i1, i2, info_d
    return u, info_d


class Prepared:
    """Algorithm 1 split in two: the constructor does the precomputation (Gaussian
    sum, Taylor coefficients, kernel tensor); run() does the actual computation.
    The paper times only the latter."""

    def __init__(self, kernel: str, n, L: float, **kw):
        self.params = make_params(kernel, n, L, **kw)
        self.shape = tuple(self.params.n[a] for a in range(self.params.d))[::-1]
        info = Info()
        self._h = lib().orc_prepare(ctypes.byref(self.params), ctypes.byref(info))
        if not self._h:
            raise RuntimeError("oracle prepare failed (bad arguments or no Gaussian sum)")
        self.info = {"S": info.S, "nterms": info.nterms, "gs_err": info.gs_err, "c0": info.c0, "c2": info.c2}

    def run(self, rho: np.ndarray) -> np.ndarray:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        if rho.shape != self.shape:
            raise ValueError(f"rho must have shape {self.shape}")
        u = np.zeros_like(rho)
        if lib().orc_run(self._h, _ptr(rho), _ptr(u), None, None) != 0:
            raise RuntimeError("oracle run failed")
        return u

    def __del__(self):
        try:
            if self._h:
                lib().orc_free_prepared(self._h)
                self._h = None
        except Exception:
            pass


def max_threads() -> int:
    return lib().orc_max_threads()


def hartree(kernel: str, psi: np.ndarray, L: float, **kw):
    """Energy E = 1/2 h^d <rho, U*rho> with rho = |psi|^2, and its gradient with
    respect to psi in PyTorch's convention for real losses (dE/dRe + i dE/dIm):
    2 h^d u psi, the operator being symmetric."""
    rho = np.abs(psi) ** 2
    u, info = apply(kernel, rho, L, **kw)
    d = rho.ndim
    h = np.prod([2.0 * L / s for s in rho.shape])
    E = 0.5 * h * float(np.sum(rho * u))
    grad = 2.0 * h * u * psi
    return E, grad, u
