"""Seeded synthetic densities shaped like the paper's test problems.

This module holds no arithmetic of the method: it only builds grids and
Gaussian-mixture densities, so both the CUDA path and the CPU oracle can be fed
the same arrays.  The paper measures only analytic Gaussian densities
(Examples 1-5 of Sec. 4), so there is no dataset to stand in for.

Grid of Sec. 2.1: x_j = -L + j h, h = 2L/n, j = 1..n; array index i = j - 1.
Arrays are C-ordered with x fastest: [z][y][x] in 3D, [y][x] in 2D.
A Gaussian is a * exp(-sum_i ((x_i - c_i) / s_i)^2), the e^{-|x|^2/sigma^2}
convention of Sec. 4.  Parameters are drawn with numpy's PCG64 in the order
centre (d values), widths (d values), amplitude, one Gaussian after another.
"""
from __future__ import annotations

import numpy as np

SEED_MIX3D = 20150104
SEED_MIX2D = 20150105
SEED_BATCH = 20150106
SEED_PSI = 20150107


def grid_1d(n: int, L: float) -> np.ndarray:
    h = 2.0 * L / n
    return -L + (np.arange(n) + 1.0) * h


def mesh(n, L):
    """Coordinate arrays (X, Y[, Z]) on the grid, each shaped like rho.  L is the
    half-width of every axis, or a sequence of per-axis half-widths (x first)."""
    if isinstance(n, int):
        raise TypeError("n must be a tuple (nx, ny[, nz])")
    Ls = list(L) if hasattr(L, "__len__") else [L] * len(n)
    axes = [grid_1d(m, a) for m, a in zip(n, Ls)]
    # meshgrid with 'ij' on reversed axes gives [z][y][x] ordering
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return tuple(grids[::-1])


def gaussian(coords, centre, widths, amp: float = 1.0) -> np.ndarray:
    e = np.zeros_like(coords[0])
    for x, c, s in zip(coords, centre, widths):
        e += ((x - c) / s) ** 2
    return amp * np.exp(-e)


def draw_mixture(rng: np.random.Generator, count: int, d: int, centre_range, width_range,
                 amp_range, isotropic: bool = False):
    params = []
    for _ in range(count):
        c = rng.uniform(centre_range[0], centre_range[1], size=d)
        if isotropic:
            s = np.full(d, rng.uniform(width_range[0], width_range[1]))
        else:
            s = rng.uniform(width_range[0], width_range[1], size=d)
        a = rng.uniform(amp_range[0], amp_range[1])
        params.append((c, s, a))
    return params


def mixture(n, L: float, params) -> np.ndarray:
    coords = mesh(n, L)
    rho = np.zeros_like(coords[0])
    for c, s, a in params:
        rho += gaussian(coords, c, s, a)
    return rho


# --- the workloads ------------------------------------------------------------

def coulomb3d_gaussian(n: int = 32, L: float = 8.0, sigma: float = 1.0) -> np.ndarray:
    """Isotropic exp(-|x|^2/sigma^2) on [-L,L]^3 (Example 1)."""
    X, Y, Z = mesh((n, n, n), L)
    return np.exp(-(X * X + Y * Y + Z * Z) / sigma ** 2)


def coulomb3d_anisotropic(n: int = 128, L: float = 12.0, gamma: float = 4.0) -> np.ndarray:
    """exp(-(x^2 + y^2 + z^2/gamma^2)) on [-L,L]^3."""
    X, Y, Z = mesh((n, n, n), L)
    return np.exp(-(X * X + Y * Y + Z * Z / gamma ** 2))


def aniso_box(d: int, L: float = 12.0, gamma: float = 4.0):
    """Box of the anisotropic rows of Sec. 4: [-L,L]^(d-1) x [-L/gamma, L/gamma]."""
    return (L,) * (d - 1) + (L / gamma,)


def aniso_gaussian(d: int, n: int, L: float = 12.0, sigma: float = 2.0, gamma: float = 4.0):
    """exp(-(|x'|^2 + gamma^2 x_d^2)/sigma^2) on aniso_box with n points per axis
    (h_d = h / gamma), the densities of the anisotropic rows of Examples 1 and 2.
    Returns (rho, box)."""
    box = aniso_box(d, L, gamma)
    C = mesh((n,) * d, box)
    r2 = sum(c * c for c in C[:-1]) + (gamma * C[-1]) ** 2
    return np.exp(-r2 / sigma ** 2), box


def mixture3d_params(seed: int = SEED_MIX3D, count: int = 8):
    rng = np.random.default_rng(seed)
    return draw_mixture(rng, count, 3, (-3.0, 3.0), (0.5, 1.5), (0.5, 2.0))


def coulomb3d_mixture(n: int = 128, L: float = 12.0, seed: int = SEED_MIX3D) -> np.ndarray:
    """Seeded 8-Gaussian mixture: centres U[-3,3]^3, per-axis widths U[0.5,1.5],
    amplitudes U[0.5,2]."""
    return mixture((n, n, n), L, mixture3d_params(seed))


def mixture2d_params(seed: int = SEED_MIX2D, count: int = 6):
    rng = np.random.default_rng(seed)
    return draw_mixture(rng, count, 2, (-4.0, 4.0), (0.5, 1.5), (0.5, 2.0), isotropic=True)


def mixture2d(n: int = 1024, L: float = 16.0, seed: int = SEED_MIX2D) -> np.ndarray:
    """Seeded 6-Gaussian isotropic mixture on [-L,L]^2: centres U[-4,4]^2,
    widths U[0.5,1.5], amplitudes U[0.5,2]."""
    return mixture((n, n), L, mixture2d_params(seed))


BATCH_SIZES = (48, 64, 96, 128, 160)


def batch_specs(count: int = 48, seed: int = SEED_BATCH, sizes=BATCH_SIZES):
    """Per-instance (n, params) for the uneven batch: n uniform in `sizes`,
    4 Gaussians each, centres U[-2,2]^3, widths U[0.5,1.5], amplitudes U[0.5,2]."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        n = int(sizes[rng.integers(0, len(sizes))])
        specs.append((n, draw_mixture(rng, 4, 3, (-2.0, 2.0), (0.5, 1.5), (0.5, 2.0))))
    return specs


def batch_densities(count: int = 48, L: float = 10.0, seed: int = SEED_BATCH, sizes=BATCH_SIZES):
    return [mixture((n, n, n), L, p) for n, p in batch_specs(count, seed, sizes)]


def psi_params(seed: int = SEED_PSI, count: int = 4, kmax: float = 2.0):
    """Gaussians (centre U[-2,2]^3, widths U[0.7,1.5], amplitude U[0.5,1.5])
    each carrying its own plane wave k_g drawn uniformly in the ball |k| <= kmax."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        c = rng.uniform(-2.0, 2.0, size=3)
        s = rng.uniform(0.7, 1.5, size=3)
        a = rng.uniform(0.5, 1.5)
        while True:
            k = rng.uniform(-kmax, kmax, size=3)
            if np.dot(k, k) <= kmax * kmax:
                break
        out.append((c, s, a, k))
    return out


def psi3d(n: int = 192, L: float = 12.0, seed: int = SEED_PSI) -> np.ndarray:
    """Complex wave function: sum_g a_g G_g(x) exp(i k_g . x)."""
    coords = mesh((n, n, n), L)
    psi = np.zeros(coords[0].shape, dtype=np.complex128)
    for c, s, a, k in psi_params(seed):
        phase = k[0] * coords[0] + k[1] * coords[1] + k[2] * coords[2]
        psi += gaussian(coords, c, s, a) * np.exp(1j * phase)
    return psi
