"""Seeded synthetic inputs: grids, relative-permittivity maps and incidence angles.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's tests.
It holds no arithmetic of the method itself (no Green's function, no operator, no
solver): it only rasterises scatterer geometries onto a cell-centred grid and draws
seeded random numbers.

Units are normalised to the background medium: wavelength lambda_b = 1, so
k_b = 2*pi; eps_b = mu_b = 1.  Every map returned here is the *relative*
permittivity eps_r(x) = eps(x)/eps_b sampled at the cell centres, as a complex128
array of shape (n2, n1) (x1 fastest), which is the layout every entry point of the
library takes.

Geometry conventions (paper Section 4 uses a uniform grid of step h over a
rectangular domain; the domain is centred at the origin as in the sinusoidal
example of Section 5):
  * cell centres are x_i = (i + 1/2) h - L/2, i = 0..n-1, L = n h;
  * a cell belongs to a scatterer when its centre lies strictly inside it.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 11044263


def rng_for(config: int, index: int = 0) -> np.random.Generator:
    """Seeded generator for workload `config`, instance `index`."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * config + index))


def cell_centres(n: int, h: float) -> np.ndarray:
    """Cell-centre coordinates (i + 1/2) h - n h / 2 for i = 0..n-1."""
    return (np.arange(n, dtype=np.float64) + 0.5) * h - 0.5 * n * h


def mesh(n1: int, n2: int, h: float):
    """(X1, X2) of shape (n2, n1): x1 varies along the last axis."""
    x1 = cell_centres(n1, h)
    x2 = cell_centres(n2, h)
    X2, X1 = np.meshgrid(x2, x1, indexing="ij")
    return X1, X2


@dataclasses.dataclass
class Problem:
    """One scattering problem: grid, eps_r map and incidence angles."""
    name: str
    n1: int
    n2: int
    h: float
    eps_r: np.ndarray           # complex128, (n2, n1)
    psi: tuple = (0.0,)         # incidence angles (radians)
    k_b: float = 2.0 * math.pi

    @property
    def N(self) -> int:
        return self.n1 * self.n2

    @property
    def unknowns(self) -> int:
        return 2 * self.N


def cylinder(n: int, side: float, radius: float, eps: complex) -> Problem:
    """Centred homogeneous circular cylinder in vacuum on an n x n grid of given side."""
    h = side / n
    X1, X2 = mesh(n, n, h)
    eps_r = np.ones((n, n), dtype=np.complex128)
    eps_r[np.hypot(X1, X2) < radius] = eps
    return Problem(f"cylinder_n{n}", n, n, h, eps_r)


def config1(n: int = 32) -> Problem:
    """Homogeneous cylinder eps_r = 4, radius 1 wavelength, square grid of side 2.5."""
    p = cylinder(n, 2.5, 1.0, 4.0 + 0.0j)
    p.name = f"cylinder eps=4 R=1 side=2.5 n={n}"
    return p


def core_shell(n: int = 512, side: float = 8.0, r_core: float = 1.5, r_shell: float = 2.5,
               eps_core: complex = -2.0 + 0.1j, eps_shell: complex = 20.0 + 0.5j) -> Problem:
    """Plasma-like core inside a dielectric shell, both centred (512^2 / side 8 by default)."""
    h = side / n
    X1, X2 = mesh(n, n, h)
    rho = np.hypot(X1, X2)
    eps_r = np.ones((n, n), dtype=np.complex128)
    eps_r[rho < r_shell] = eps_shell
    eps_r[rho < r_core] = eps_core
    return Problem(f"core-shell n={n} side={side}", n, n, h, eps_r)


def config2(n: int = 512) -> Problem:
    """Core (eps -2+0.1i, R 1.5) in shell (eps 20+0.5i, R 2.5); side 8 at h = 1/64 for n = 512."""
    return core_shell(n, side=8.0 * n / 512.0, r_core=1.5 * n / 512.0, r_shell=2.5 * n / 512.0)


def square(n: int, h: float, eps_outer: complex, eps_inner: complex | None = None) -> Problem:
    """A grid entirely filled by a square scatterer (the paper's test objects, Section 4).

    With `eps_inner` the central square of half the side holds eps_inner (the
    inhomogeneous core/shell test object).
    """
    eps_r = np.full((n, n), eps_outer, dtype=np.complex128)
    if eps_inner is not None:
        X1, X2 = mesh(n, n, h)
        a = n * h
        eps_r[(np.abs(X1) < a / 4) & (np.abs(X2) < a / 4)] = eps_inner
    return Problem(f"square n={n} eps={eps_outer}", n, n, h, eps_r)


def paper_squares(n: int = 61, h: float = 1.0 / 60.0):
    """The three test scatterers of Section 4: eps 16; -16+1.5i; 2.5+20i core in a 16 shell."""
    return [square(n, h, 16.0 + 0j), square(n, h, -16.0 + 1.5j),
            square(n, h, 16.0 + 0j, 2.5 + 20.0j)]


def _normal_cdf(x: np.ndarray) -> np.ndarray:
    from scipy.special import ndtr
    return ndtr(x)


def _gaussian_field(rng: np.random.Generator, n: int, h: float, corr: float) -> np.ndarray:
    """Unit-variance Gaussian random field with a Gaussian correlation of length `corr`."""
    white = rng.standard_normal((n, n))
    f = np.fft.fftfreq(n, d=h)
    F2, F1 = np.meshgrid(f, f, indexing="ij")
    # spectrum of the smoothing kernel exp(-d^2 / (2 corr^2))
    filt = np.exp(-2.0 * (math.pi * corr) ** 2 * (F1 ** 2 + F2 ** 2))
    g = np.real(np.fft.ifft2(np.fft.fft2(white) * filt))
    s = g.std()
    return (g - g.mean()) / (s if s > 0 else 1.0)


def sinusoidal(n: int = 233, a: float = 4.0) -> Problem:
    """Section 5's continuous-permittivity object: eps_r = 10 + 5 sin(4 pi x1 / a)
    sin(4 pi x2 / a) over the whole square domain of side a (origin at its centre), on an
    n x n grid (233 x 233 at a = 4 wavelengths: 15 points per smallest medium wavelength)."""
    h = a / n
    X1, X2 = mesh(n, n, h)
    eps_r = (10.0 + 5.0 * np.sin(4.0 * math.pi * X1 / a) * np.sin(4.0 * math.pi * X2 / a)).astype(np.complex128)
    return Problem(f"sinusoidal a={a} n={n}", n, n, h, eps_r)


def lossless_square(a_over_lambda: float, eps: float = 16.0, ppw: int = 15) -> Problem:
    """Section 5's sweep object: a homogeneous lossless square filling the domain, side a,
    at `ppw` points per medium wavelength (n = round(ppw sqrt(eps) a / lambda) + 1 cells)."""
    n = int(round(ppw * math.sqrt(eps) * a_over_lambda)) + 1
    return square(n, a_over_lambda / n, complex(eps))


BATCH_SIZES = (64, 96, 128, 192, 256, 384, 512)


def config3(count: int = 64, sizes=BATCH_SIZES, h: float = 1.0 / 60.0, n_angles: int = 8):
    """Batched workload: `count` Gaussian-random scatterers masked to random ellipses.

    Re eps_r = 1 + 15 Phi(g1), Im eps_r = Phi(g2) inside the ellipse (g1, g2
    independent unit-variance fields of correlation length 0.3), eps_r = 1 outside;
    incidence angles psi_j = 2 pi j / n_angles.
    """
    out = []
    for i in range(count):
        rng = rng_for(3, i)
        n = int(rng.choice(np.asarray(sizes)))
        side = n * h
        g1 = _gaussian_field(rng, n, h, 0.3)
        g2 = _gaussian_field(rng, n, h, 0.3)
        eps_in = (1.0 + 15.0 * _normal_cdf(g1)) + 1j * _normal_cdf(g2)
        c1, c2 = rng.uniform(-0.1, 0.1, size=2) * side
        a, b = rng.uniform(0.25, 0.45, size=2) * side
        th = rng.uniform(0.0, math.pi)
        X1, X2 = mesh(n, n, h)
        u = (X1 - c1) * math.cos(th) + (X2 - c2) * math.sin(th)
        v = -(X1 - c1) * math.sin(th) + (X2 - c2) * math.cos(th)
        inside = (u / a) ** 2 + (v / b) ** 2 < 1.0
        eps_r = np.where(inside, eps_in, 1.0 + 0j).astype(np.complex128)
        psi = tuple(2.0 * math.pi * j / n_angles for j in range(n_angles))
        out.append(Problem(f"gaussian-ellipse #{i} n={n}", n, n, h, eps_r, psi))
    return out


def config4_field(index: int, n: int = 128, h: float = 1.0 / 60.0, corr: float = 0.3,
                  min_abs: float = 0.25, re_lo: float = -4.0) -> Problem:
    """Learned-preconditioner workload: a seeded Gaussian random permittivity field over the
    whole n x n grid, Re eps_r = re_lo + (16 - re_lo) Phi(g1) in [re_lo, 16] (re_lo = -4 by
    default), Im eps_r = Phi(g2) in [0, 1] (g1, g2 independent unit-variance fields of
    correlation length `corr`), values with |eps_r| < min_abs pushed out to |eps_r| = min_abs
    (the existence condition eps != 0), and a random incidence angle.  index selects the
    seed (training and held-out sets use disjoint ranges)."""
    rng = rng_for(4, index)
    g1 = _gaussian_field(rng, n, h, corr)
    g2 = _gaussian_field(rng, n, h, corr)
    eps = (re_lo + (16.0 - re_lo) * _normal_cdf(g1)) + 1j * _normal_cdf(g2)
    a = np.abs(eps)
    small = a < min_abs
    eps[small] = np.where(a[small] > 0, eps[small] / np.where(a[small] > 0, a[small], 1.0) * min_abs, min_abs)
    psi = float(rng.uniform(0.0, 2.0 * math.pi))
    return Problem(f"random field #{index} n={n}", n, n, h, eps.astype(np.complex128), (psi,))


def smooth_random_vector(rng: np.random.Generator, n1: int, n2: int, h: float, corr: float = 0.1) -> np.ndarray:
    """Random complex (E1, E2) field of shape (2, n2, n1) with Gaussian correlation of length
    `corr` (in wavelengths) and unit root-mean-square value."""
    assert n1 == n2
    parts = [_gaussian_field(rng, n1, h, corr) for _ in range(4)]
    v = np.stack([parts[0] + 1j * parts[1], parts[2] + 1j * parts[3]]) / math.sqrt(2.0)
    return v.astype(np.complex128)


CFG5_EPS = (-6.0 + 0.5j, 2.0 + 0j, 9.0 + 0j, 30.0 + 1.0j)


def random_cylinders(n: int = 2048, side: float = 32.0, count: int = 400,
                     rmin: float = 0.2, rmax: float = 0.6, eps_set=CFG5_EPS, seed_index: int = 0):
    """`count` seeded cylinders (later ones overwrite earlier ones) on an n x n grid."""
    rng = rng_for(5, seed_index)
    h = side / n
    x = cell_centres(n, h)
    eps_r = np.ones((n, n), dtype=np.complex128)
    half = side / 2
    for _ in range(count):
        R = rng.uniform(rmin, rmax)
        c1, c2 = rng.uniform(-half + R, half - R, size=2)
        e = eps_set[int(rng.integers(len(eps_set)))]
        i1 = np.nonzero(np.abs(x - c1) < R)[0]
        i2 = np.nonzero(np.abs(x - c2) < R)[0]
        if i1.size == 0 or i2.size == 0:
            continue
        sub2, sub1 = np.meshgrid(x[i2], x[i1], indexing="ij")
        m = np.hypot(sub1 - c1, sub2 - c2) < R
        blk = eps_r[i2[0]:i2[-1] + 1, i1[0]:i1[-1] + 1]
        blk[m] = e
    return Problem(f"random cylinders n={n} count={count}", n, n, h, eps_r)


def random_field(rng: np.random.Generator, n1: int, n2: int, lo: float = 1.0, hi: float = 16.0,
                 loss: float = 1.0) -> np.ndarray:
    """Cell-wise independent random eps_r (for operator parity tests on ragged grids)."""
    re = rng.uniform(lo, hi, size=(n2, n1))
    im = rng.uniform(0.0, loss, size=(n2, n1))
    return (re + 1j * im).astype(np.complex128)


def random_vector(rng: np.random.Generator, n1: int, n2: int) -> np.ndarray:
    """Random complex (E1, E2) field of shape (2, n2, n1)."""
    return (rng.standard_normal((2, n2, n1)) + 1j * rng.standard_normal((2, n2, n1))).astype(np.complex128)
