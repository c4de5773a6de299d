"""Seeded synthetic inputs for the Crank-Nicolson / HIF-PCG workloads.

This module only draws random numbers and evaluates closed-form fields on the
grid.  It holds none of the method's arithmetic (no stencil, no factorization,
no solver), so both the CPU oracle and the CUDA path may take their inputs from
it.

Grid convention (Sec. 2 of the paper): the unit cube (0,1)^d carries
``n = 1/h = 2^L * m`` intervals per axis.  The unknowns sit on the interior
nodes ``x_j = h*j`` with ``1 <= j_axis <= n-1``, so ``N = (n-1)^d``.  Arrays
are C-ordered with the *last* axis being x (fastest varying):

* nodal coefficient ``a``: shape ``(n+1,)*d`` (boundary nodes included),
* interior field ``u``: shape ``(n-1,)*d``; flattened, DOF index
  ``j_1-1 + (n-1)*(j_2-1) [+ (n-1)^2*(j_3-1)]``.

All fields are float64 numpy arrays.  The generators follow the workload
recipes: Gaussian random fields filtered in Fourier space, lognormal
coefficients with a prescribed contrast, the sine-mode and Gaussian-bump
initial conditions of the paper's examples (Sec. 3, Eq. 2d_u0 and 3d_u0).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "node_coords",
    "interior_coords",
    "grf",
    "lognormal_coefficient",
    "gaussian_bump_u0",
    "sine_modes_u0",
    "snap_side",
    "config_heat2d_63",
    "config_fisher2d_1023",
    "config_heat3d_127",
    "config_batched",
    "small_variable_2d",
    "gaussian_bumps_coefficient",
    "paper_heat2d",
    "paper_logistic2d",
    "paper_heat3d",
]


def node_coords(n: int, dim: int) -> list[np.ndarray]:
    """Coordinates of the (n+1)^dim nodes, one broadcastable array per axis.

    Returned in the order (x, y[, z]); array axis -1 is x.
    """
    t = np.arange(n + 1, dtype=np.float64) / n
    out = []
    for ax in range(dim):
        shape = [1] * dim
        shape[dim - 1 - ax] = n + 1
        out.append(t.reshape(shape))
    return out


def interior_coords(n: int, dim: int) -> list[np.ndarray]:
    """Coordinates of the (n-1)^dim interior nodes (x, y[, z])."""
    t = np.arange(1, n, dtype=np.float64) / n
    out = []
    for ax in range(dim):
        shape = [1] * dim
        shape[dim - 1 - ax] = n - 1
        out.append(t.reshape(shape))
    return out


def grf(rng: np.random.Generator, n: int, dim: int, corr_len: float) -> np.ndarray:
    """Zero-mean Gaussian random field on the (n+1)^dim node grid.

    White noise filtered in Fourier space by exp(-|k|^2 corr_len^2 / 2), with
    wavenumbers in radians per unit length of the unit domain.
    """
    shape = (n + 1,) * dim
    w = rng.standard_normal(shape)
    spec = np.fft.fftn(w)
    k2 = np.zeros(shape)
    for ax in range(dim):
        k = 2.0 * np.pi * np.fft.fftfreq(n + 1, d=1.0 / n)
        s = [1] * dim
        s[ax] = n + 1
        k2 = k2 + (k.reshape(s)) ** 2
    g = np.real(np.fft.ifftn(spec * np.exp(-0.5 * k2 * corr_len * corr_len)))
    return g - g.mean()


def lognormal_coefficient(g: np.ndarray, contrast: float) -> np.ndarray:
    """a = exp(g * ln(C) / (max g - min g)) so that max(a)/min(a) = C."""
    span = float(g.max() - g.min())
    if span == 0.0:
        return np.ones_like(g)
    return np.exp(g * (math.log(contrast) / span))


def gaussian_bump_u0(n: int, dim: int, sigma2: float = 0.05, center: float = 0.5,
                     amplitude: float | None = None) -> np.ndarray:
    """Gaussian bump on the interior nodes (paper Example 2, Eq. 2d_u0).

    Default amplitude 2/(3 sqrt(2 pi sigma^2)) as printed for the 2D logistic
    example.
    """
    if amplitude is None:
        amplitude = 2.0 / (3.0 * math.sqrt(2.0 * math.pi * sigma2))
    xs = interior_coords(n, dim)
    r2 = sum((x - center) ** 2 for x in xs)
    return amplitude * np.exp(-r2 / sigma2)


def sine_modes_u0(n: int, dim: int, modes, rng: np.random.Generator | None = None,
                  noise: float = 0.0) -> np.ndarray:
    """Sum of sine modes prod_axis sin(k_axis pi x_axis) plus uniform noise."""
    xs = interior_coords(n, dim)
    u = np.zeros((n - 1,) * dim)
    for mode in modes:
        term = np.ones((n - 1,) * dim)
        for ax, k in enumerate(mode):
            term = term * np.sin(k * math.pi * xs[ax])
        u = u + term
    if noise > 0.0:
        assert rng is not None
        u = u + rng.uniform(-noise, noise, size=u.shape)
    return u


def snap_side(side: float, leafs=range(8, 17)) -> tuple[int, int, int]:
    """Snap an interior side length s to the nearest (2^L m - 1).

    Returns (n, m, L) with n = 2^L m, m in ``leafs`` and L >= 1; the paper
    needs n = 2^L m (Sec. 2), uneven requested sizes are rounded to the
    closest admissible one (ties to the smaller n).
    """
    best = None
    for m in leafs:
        for L in range(1, 16):
            n = (1 << L) * m
            d = abs((n - 1) - side)
            key = (d, n)
            if best is None or key < best[0]:
                best = (key, (n, m, L))
    return best[1]


@dataclass
class Workload:
    """One Crank-Nicolson problem instance."""

    name: str
    dim: int
    n: int
    leaf: int
    levels: int
    dt: float
    eps: float
    a_nodes: np.ndarray
    u0: np.ndarray
    reaction: tuple[int, float, float] = (0, 0.0, 0.0)  # (kind, k1, k2); kind 1 = logistic
    steps: int = 10
    tol: float = 1e-10
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return (self.n - 1) ** self.dim


def config_heat2d_63(seed: int = 0) -> Workload:
    """2D heat, a = 1, 63x63 interior (n=64, leaf 8, L=3), dt=1e-2, eps=1e-6."""
    n, m, L = 64, 8, 3
    rng = np.random.default_rng(seed)
    u0 = sine_modes_u0(n, 2, [(1, 1), (2, 3), (5, 2)], rng=rng, noise=0.1)
    return Workload("heat2d_63", 2, n, m, L, 1e-2, 1e-6, np.ones((n + 1,) * 2), u0,
                    (0, 0.0, 0.0), steps=10)


def config_fisher2d_1023(eps: float = 1e-6, seed: int = 1) -> Workload:
    """2D Fisher-KPP, lognormal a (GRF corr 0.05, contrast 1e4), 1023^2, dt=1."""
    n, m, L = 1024, 16, 6
    rng = np.random.default_rng(seed)
    a = lognormal_coefficient(grf(rng, n, 2, 0.05), 1e4)
    u0 = gaussian_bump_u0(n, 2)
    return Workload("fisher2d_1023", 2, n, m, L, 1.0, eps, a, u0, (1, 1.0, 1.0), steps=100)


def config_heat3d_127(seed: int = 2) -> Workload:
    """3D heat, lognormal a (contrast 1e3), 127^3 (n=128, leaf 8, L=4), dt=0.1."""
    n, m, L = 128, 8, 4
    rng = np.random.default_rng(seed)
    a = lognormal_coefficient(grf(rng, n, 3, 0.05), 1e3)
    g = grf(np.random.default_rng(seed + 1), n, 3, 0.1)[1:-1, 1:-1, 1:-1]
    u0 = g / np.abs(g).max()
    return Workload("heat3d_127", 3, n, m, L, 0.1, 1e-4, a, u0, (0, 0.0, 0.0), steps=50)


def config_batched(count: int = 256, seed0: int = 1000, lo: float = 63, hi: float = 511):
    """Uneven 2D reaction-diffusion problems (side log-uniform, snapped)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        side = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        n, m, L = snap_side(side)
        a = lognormal_coefficient(grf(rng, n, 2, 0.05), 1e3)
        dt = math.exp(rng.uniform(math.log(1e-2), math.log(1.0)))
        u0 = gaussian_bump_u0(n, 2)
        out.append(Workload(f"batched_{i}", 2, n, m, L, dt, 1e-6, a, u0, (1, 1.0, 1.0),
                            steps=20, meta={"side_drawn": side}))
    return out


def config_serving(count2d: int = 48, count3d: int = 16, seed0: int = 2000):
    """Serving mix of resident operators: 2D operators with side log-uniform in
    [255, 2047] (snapped, leaf 16) and 3D operators with side drawn uniformly
    from {63, 95, 127} (snapped: leaf 8, 12, 8); operator i uses seed
    seed0 + i.  Lognormal a (GRF corr 0.05, contrast 1e3), dt log-uniform in
    [1e-2, 1], r = u(1-u), the bump u0; eps 1e-6 in 2D and 1e-4 in 3D (the
    3D benchmark's tolerance)."""
    out = []
    for i in range(count2d + count3d):
        rng = np.random.default_rng(seed0 + i)
        if i < count2d:
            dim = 2
            side = math.exp(rng.uniform(math.log(255), math.log(2047)))
            n, m, L = snap_side(side, leafs=(16,))
            eps = 1e-6
        else:
            dim = 3
            side = float(rng.choice([63, 95, 127]))
            n, m, L = snap_side(side, leafs=(8, 12))
            eps = 1e-4
        a = lognormal_coefficient(grf(rng, n, dim, 0.05), 1e3)
        dt = math.exp(rng.uniform(math.log(1e-2), math.log(1.0)))
        out.append(Workload(f"serving_{i}", dim, n, m, L, dt, eps, a, gaussian_bump_u0(n, dim),
                            (1, 1.0, 1.0), steps=1, meta={"side_drawn": side}))
    return out


def small_variable_2d(n: int = 32, m: int = 8, seed: int = 7, contrast: float = 1e2,
                      dt: float = 1.0, eps: float = 1e-6, dim: int = 2,
                      corr_len: float = 0.1) -> Workload:
    """A small variable-coefficient problem of any admissible size (tests)."""
    L = int(round(math.log2(n // m)))
    assert (1 << L) * m == n
    rng = np.random.default_rng(seed)
    a = lognormal_coefficient(grf(rng, n, dim, corr_len), contrast)
    u0 = gaussian_bump_u0(n, dim)
    return Workload(f"small{dim}d_{n}", dim, n, m, L, dt, eps, a, u0, (1, 1.0, 1.0), steps=3)


def gaussian_bumps_coefficient(rng: np.random.Generator, n: int, dim: int, count: int,
                               sigma2: float, lo: float, hi: float) -> np.ndarray:
    """Sum of ``count`` Gaussian bumps at uniform random centres, mapped affinely
    onto [lo, hi] (paper Eqs. 2d_coeff / 3d_coeff; min -> lo, max -> hi)."""
    centres = rng.uniform(0.0, 1.0, size=(count, dim))
    t = np.arange(n + 1, dtype=np.float64) / n
    # each bump is a product of one Gaussian per axis: E[ax][c, i] at coordinate t_i
    E = [np.exp(-((t[None, :] - centres[:, ax, None]) ** 2) / sigma2) for ax in range(dim)]
    if dim == 2:
        s = E[1].T @ E[0]  # s[y, x] = sum_c E_y[c, y] E_x[c, x]
    else:
        zy = (E[2][:, :, None] * E[1][:, None, :]).reshape(count, -1)
        s = (zy.T @ E[0]).reshape((n + 1,) * 3)
    smin, smax = float(s.min()), float(s.max())
    return lo + (s - smin) * ((hi - lo) / (smax - smin))


def paper_heat2d(n: int, leaf: int, eps: float, seed: int = 0) -> Workload:
    """Paper Example 1 (2D heat) generator: 100 bumps (sigma_2^2 = 0.005) on
    [0.1, 10], u0 = two Gaussians at (0.35, 0.35) and (0.65, 0.65) with
    sigma^2 = 0.05, dt = h (reading of the printed "dt = dx = 1/N")."""
    L = int(round(math.log2(n // leaf)))
    rng = np.random.default_rng(seed)
    a = gaussian_bumps_coefficient(rng, n, 2, 100, 0.005, 0.1, 10.0)
    xs = interior_coords(n, 2)
    u0 = sum(np.exp(-sum((x - c) ** 2 for x in xs) / 0.05) for c in (0.35, 0.65))
    return Workload(f"paper_heat2d_{n - 1}", 2, n, leaf, L, 1.0 / n, eps, a, u0,
                    (0, 0.0, 0.0), steps=100, tol=1e-12)


def paper_logistic2d(n: int, leaf: int, eps: float, seed: int = 0) -> Workload:
    """Paper Example 2 (2D logistic) generator: the coefficient of Example 1,
    u0 the bump of Eq. 2d_u0 (c = 0.5, sigma^2 = 0.05), k1 = 1, k2 = 10,
    dt = h as in Example 1."""
    L = int(round(math.log2(n // leaf)))
    rng = np.random.default_rng(seed)
    a = gaussian_bumps_coefficient(rng, n, 2, 100, 0.005, 0.1, 10.0)
    u0 = gaussian_bump_u0(n, 2)
    return Workload(f"paper_logistic2d_{n - 1}", 2, n, leaf, L, 1.0 / n, eps, a, u0,
                    (1, 1.0, 10.0), steps=100, tol=1e-12)


def paper_heat3d(n: int, leaf: int, eps: float, seed: int = 0,
                 logistic: bool = False) -> Workload:
    """Paper Example 1 in 3D (and Example 2 in 3D with ``logistic``): bumps
    with sigma_2^2 = 0.005 on [0.05, 20] (1000 of them; 200 for the logistic
    case), u0 the Gaussian of Eq. 3d_u0 at c = 0.5 with sigma^2 = 0.05 (times
    (2 pi sigma)^{-3/2} for the logistic case), dt = 0.1 h."""
    L = int(round(math.log2(n // leaf)))
    rng = np.random.default_rng(seed)
    a = gaussian_bumps_coefficient(rng, n, 3, 200 if logistic else 1000, 0.005, 0.05, 20.0)
    amp = (2.0 * math.pi * math.sqrt(0.05)) ** -1.5 if logistic else 1.0
    u0 = gaussian_bump_u0(n, 3, amplitude=amp)
    name = "paper_logistic3d" if logistic else "paper_heat3d"
    return Workload(f"{name}_{n - 1}", 3, n, leaf, L, 0.1 / n, eps, a, u0,
                    (1, 1.0, 10.0) if logistic else (0, 0.0, 0.0), steps=100, tol=1e-12)
