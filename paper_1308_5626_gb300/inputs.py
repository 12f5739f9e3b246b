"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle.

This module holds workload definitions and random-number draws only.  It contains none
of the method's arithmetic: no finite-difference weights, no operator, no solver.  Every
draw uses numpy's PCG64 generator with the seed stated beside the workload, so both sides
of a parity test see bit-identical inputs.

Workloads (all periodic on [0, 2*pi)^d, h = 2*pi/n per direction, x fastest):

* ``c1``  1D advection-diffusion u_t = a u_x + nu u_xx, 4th-order central FD, n = 1024,
  a = 1, nu = 0.01, dt = 10 h / a (advective CFL 10), restart m = 30, band b = 2,
  20 implicit steps, tol 1e-10; u^0 = sum of 16 sines with N(0,1) amplitudes and
  U[0, 2pi) phases (seed 1).
* ``c2``  2D anisotropic advection-diffusion, 6th-order central FD (13-point cross),
  1024 x 1024; a_x, a_y ~ U[0.5, 2], nu_x, nu_y ~ U[0.5, 2] * 1e-3; dt = 20 h / max(a);
  m = 40, b = 4, 10 steps; u^0 a Gaussian random field with power ~ |k|^-2, zero mean,
  unit RMS (seed 2).
* ``c3``  3D diffusion plus hyperdiffusion u_t = sum_i alpha_i u_{x_i x_i}
  - beta sum_i u_{x_i x_i x_i x_i}, 8th-order central FD (31-point cross), 256^3;
  alpha_i ~ U[0.5, 2], beta = mean(alpha) (h/pi)^2; dt = 100 / rho(L) with rho the
  spectral radius of the discrete operator (each side evaluates it from its own
  stencil); m = 50, b = 3, 5 steps; u^0 white noise low-passed to |k| < 32, unit RMS
  (seed 3).

Small variants (same recipe, smaller grids) serve the parity tests.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class Term:
    """One term alpha * d^k u / dx_dir^k of the linear operator (Eq. 1)."""

    k: int
    dir: int
    alpha: float


@dataclasses.dataclass
class Workload:
    name: str
    shape: Tuple[int, ...]          # (nx,) or (nx, ny) or (nx, ny, nz); x fastest in memory
    order: int                      # accuracy order of every central difference
    terms: List[Term]
    b: int                          # band half-width of the preconditioner N
    m: int                          # GMRES restart length
    steps: int                      # implicit steps in the time series
    tol: float                      # relative residual tolerance of one step
    dt: Optional[float]             # None: derived from rho(L) * dt = rho_dt
    rho_dt: Optional[float]         # spectral-radius target when dt is None
    u0: np.ndarray                  # flattened, x fastest, float64
    seed: int

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    @property
    def h(self) -> Tuple[float, ...]:
        return tuple(TWO_PI / s for s in self.shape)

    def with_dt(self, rho: float) -> float:
        """Time step for a spectral-radius rule: dt = rho_dt / rho(L)."""
        if self.dt is not None:
            return self.dt
        return self.rho_dt / rho


# --------------------------------------------------------------------------------------
# initial data
# --------------------------------------------------------------------------------------

def sines_1d(n: int, count: int, rng: np.random.Generator) -> np.ndarray:
    """u(x) = sum_{j=1..count} A_j sin(j x + phi_j), A_j ~ N(0,1), phi_j ~ U[0, 2pi)."""
    amp = rng.standard_normal(count)
    phase = rng.uniform(0.0, TWO_PI, count)
    x = np.arange(n) * (TWO_PI / n)
    u = np.zeros(n)
    for j in range(count):
        u += amp[j] * np.sin((j + 1) * x + phase[j])
    return u


def _wavenumbers(shape_zyx: Sequence[int]) -> List[np.ndarray]:
    return [np.fft.fftfreq(s, d=1.0 / s) for s in shape_zyx]


def gaussian_random_field(shape: Tuple[int, ...], rng: np.random.Generator,
                          power: float = -2.0) -> np.ndarray:
    """Zero-mean, unit-RMS Gaussian random field whose power spectrum is ~ |k|^power.

    White noise is filtered in Fourier space by |k|^(power/2) (k != 0); the mean mode is
    removed.  ``shape`` is (nx, ny, ...) with x fastest; the result is flattened.
    """
    zyx = tuple(reversed(shape))
    white = rng.standard_normal(zyx)
    ks = _wavenumbers(zyx)
    grids = np.meshgrid(*ks, indexing="ij")
    k2 = np.zeros(zyx)
    for g in grids:
        k2 = k2 + g * g
    filt = np.zeros(zyx)
    nz = k2 > 0
    filt[nz] = k2[nz] ** (power / 4.0)
    u = np.real(np.fft.ifftn(np.fft.fftn(white) * filt))
    u -= u.mean()
    u /= math.sqrt(np.mean(u * u))
    return u.reshape(-1).copy()


def lowpass_noise(shape: Tuple[int, ...], rng: np.random.Generator, kmax: float) -> np.ndarray:
    """White N(0,1) noise keeping only integer wavenumbers with |k| < kmax, unit RMS."""
    zyx = tuple(reversed(shape))
    white = rng.standard_normal(zyx)
    ks = _wavenumbers(zyx)
    grids = np.meshgrid(*ks, indexing="ij")
    k2 = np.zeros(zyx)
    for g in grids:
        k2 = k2 + g * g
    mask = (k2 < kmax * kmax).astype(np.float64)
    u = np.real(np.fft.ifftn(np.fft.fftn(white) * mask))
    u /= math.sqrt(np.mean(u * u))
    return u.reshape(-1).copy()


# --------------------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------------------

def c1(n: int = 1024) -> Workload:
    """1D periodic advection-diffusion, 4th order, CFL 10 (seed 1)."""
    rng = np.random.default_rng(1)
    a, nu = 1.0, 0.01
    h = TWO_PI / n
    u0 = sines_1d(n, 16, rng)
    return Workload("c1_1d_adv_diff_%d" % n, (n,), 4,
                    [Term(1, 0, a), Term(2, 0, nu)], b=2, m=30, steps=20, tol=1e-10,
                    dt=10.0 * h / a, rho_dt=None, u0=u0, seed=1)


def c2(nx: int = 1024, ny: Optional[int] = None) -> Workload:
    """2D periodic anisotropic advection-diffusion, 6th order, CFL 20 (seed 2)."""
    ny = nx if ny is None else ny
    rng = np.random.default_rng(2)
    a = rng.uniform(0.5, 2.0, 2)
    nu = rng.uniform(0.5, 2.0, 2) * 1e-3
    u0 = gaussian_random_field((nx, ny), rng, power=-2.0)
    h = TWO_PI / nx
    terms = [Term(1, 0, float(a[0])), Term(1, 1, float(a[1])),
             Term(2, 0, float(nu[0])), Term(2, 1, float(nu[1]))]
    return Workload("c2_2d_aniso_adv_diff_%dx%d" % (nx, ny), (nx, ny), 6, terms,
                    b=4, m=40, steps=10, tol=1e-10, dt=20.0 * h / float(a.max()),
                    rho_dt=None, u0=u0, seed=2)


def c3(n: int = 256, kmax: float = 32.0, with_u0: bool = True) -> Workload:
    """3D periodic diffusion + hyperdiffusion, 8th order, rho(L) dt = 100 (seed 3).
    with_u0=False skips the initial field (u0 = None) for uses that need only the operator."""
    rng = np.random.default_rng(3)
    alpha = rng.uniform(0.5, 2.0, 3)
    h = TWO_PI / n
    beta = float(alpha.mean()) * (h / math.pi) ** 2
    u0 = lowpass_noise((n, n, n), rng, min(kmax, n / 2.0)) if with_u0 else None
    terms = [Term(2, d, float(alpha[d])) for d in range(3)] + \
            [Term(4, d, -beta) for d in range(3)]
    return Workload("c3_3d_diff_hyperdiff_%d^3" % n, (n, n, n), 8, terms,
                    b=3, m=50, steps=5, tol=1e-10, dt=None, rho_dt=100.0, u0=u0, seed=3)


def c5(n: int = 512) -> Tuple[Workload, np.ndarray]:
    """2D periodic anisotropic diffusion u_t = a_x u_xx + a_y u_yy, 6th order, rho(L) dt = 10,
    10 steps (seed 5): the true coefficients a ~ U[0.5, 2] 1e-3 define the workload; the
    returned perturbation factors (1 + 0.1 U[-1, 1]) give the coefficients at which a loss
    against a target made with the true ones is differentiated."""
    rng = np.random.default_rng(5)
    a = rng.uniform(0.5, 2.0, 2) * 1e-3
    u0 = gaussian_random_field((n, n), rng, power=-2.0)
    factors = 1.0 + 0.1 * rng.uniform(-1.0, 1.0, 2)
    terms = [Term(2, 0, float(a[0])), Term(2, 1, float(a[1]))]
    w = Workload("c5_2d_aniso_diff_%dx%d" % (n, n), (n, n), 6, terms, b=4, m=30, steps=10, tol=1e-12,
                 dt=None, rho_dt=10.0, u0=u0, seed=5)
    return w, factors


def c4_instance(i: int, e_range: Tuple[int, int] = (10, 18)) -> Workload:
    """Instance i of the batched workload (seed 4 + i): a coin picks the 1D form of c1 or the
    2D form of c2; n = 2^e with e uniform over the integers of e_range (log-uniform sizes; a
    2D grid splits as n_x = 2^ceil(e/2), n_y = 2^floor(e/2)); accuracy order from
    {2, 4, 6, 8}; b from 1..4; CFL ~ U[1, 20]; restart 30; tolerance 1e-8."""
    rng = np.random.default_rng(4 + i)
    two_d = bool(rng.integers(0, 2))
    e = int(rng.integers(e_range[0], e_range[1] + 1))
    order = int(rng.choice([2, 4, 6, 8]))
    b = int(rng.integers(1, 5))
    cfl = float(rng.uniform(1.0, 20.0))
    return _c4_build(rng, "c4_%d" % i, two_d, e, order, b, cfl, 4 + i)


def c4_spec(two_d: bool, e: int, order: int, b: int, cfl: float, seed: int) -> Workload:
    """A batched-workload instance with its size, order, band and CFL chosen by the caller
    (the coefficients and u^0 drawn as in c4_instance from the given seed): the parity tests
    pick instances that span the batch's ranges."""
    rng = np.random.default_rng(seed)
    return _c4_build(rng, "c4s%d" % seed, bool(two_d), int(e), int(order), int(b), float(cfl), seed)


def _c4_build(rng, tag, two_d, e, order, b, cfl, seed) -> Workload:
    if two_d:
        nx, ny = 2 ** ((e + 1) // 2), 2 ** (e // 2)
        a = rng.uniform(0.5, 2.0, 2)
        nu = rng.uniform(0.5, 2.0, 2) * 1e-3
        terms = [Term(1, 0, float(a[0])), Term(1, 1, float(a[1])),
                 Term(2, 0, float(nu[0])), Term(2, 1, float(nu[1]))]
        u0 = gaussian_random_field((nx, ny), rng, power=-2.0)
        shape, dt = (nx, ny), cfl * (TWO_PI / nx) / float(a.max())
    else:
        n = 2 ** e
        terms = [Term(1, 0, 1.0), Term(2, 0, 0.01)]
        u0 = sines_1d(n, 16, rng)
        shape, dt = (n,), cfl * (TWO_PI / n)
    return Workload("%s_%s" % (tag, "x".join(str(s) for s in shape)), shape, order, terms, b=b, m=30,
                    steps=10, tol=1e-8, dt=dt, rho_dt=None, u0=u0, seed=seed)


WORKLOADS = {"c1": c1, "c2": c2, "c3": c3}


# --------------------------------------------------------------------------------------
# fixtures for the kernels taken one at a time
# --------------------------------------------------------------------------------------

def random_band(n: int, b: int, seed: int, dominance: float = 1.5) -> np.ndarray:
    """Random banded matrix in row-major band storage band[i, p] = N(i, i + p - b).

    Off-diagonals ~ U[-1, 1]; the diagonal is dominance * (sum of |off-diagonals|) + 1
    with a random sign, so every leading block is nonsingular.  Entries whose column
    falls outside [0, n) are zero.
    """
    rng = np.random.default_rng(seed)
    band = rng.uniform(-1.0, 1.0, (n, 2 * b + 1))
    for p in range(2 * b + 1):
        off = p - b
        lo = max(0, -off)
        hi = min(n, n - off)
        band[:lo, p] = 0.0
        band[hi:, p] = 0.0
    band[:, b] = 0.0
    diag = dominance * np.abs(band).sum(axis=1) + 1.0
    sign = np.where(rng.uniform(0.0, 1.0, n) < 0.5, -1.0, 1.0)
    band[:, b] = sign * diag
    return band


def random_cyclic_band(n: int, b: int, seed: int, dominance: float = 1.5) -> np.ndarray:
    """Random cyclic band (band[i, p] = N(i, (i + p - b) mod n)): as ``random_band`` but
    with every cell filled, the wrapped corner cells of the first and last b rows included."""
    rng = np.random.default_rng(seed)
    band = rng.uniform(-1.0, 1.0, (n, 2 * b + 1))
    band[:, b] = 0.0
    diag = dominance * np.abs(band).sum(axis=1) + 1.0
    sign = np.where(rng.uniform(0.0, 1.0, n) < 0.5, -1.0, 1.0)
    band[:, b] = sign * diag
    return band


def random_pd_part_band(n: int, b: int, seed: int, skew: float = 3.0) -> np.ndarray:
    """Banded matrix with positive-definite symmetric part but no diagonal dominance.

    N = S + K with S = I + (banded symmetric positive semi-definite Laplacian-like part)
    and K a banded skew-symmetric part scaled by ``skew``: the shape of I - dt*L for an
    advection-dominated implicit step.  Band storage as in ``random_band``.
    """
    rng = np.random.default_rng(seed)
    band = np.zeros((n, 2 * b + 1))
    band[:, b] = 1.0
    for off in range(1, b + 1):
        w = rng.uniform(0.2, 1.0, n)          # symmetric part: w * (e_i - e_j)(e_i - e_j)^T
        k = rng.uniform(-1.0, 1.0, n) * skew  # skew part
        # pair (i, j = i + off) for i < n - off; row j receives its share before row j's own
        # pair (j, j + off) adds to it, the order of a loop over i
        wi, ki = w[:n - off], k[:n - off]
        band[off:, b] += wi
        band[:n - off, b] += wi
        band[:n - off, b + off] += -wi + ki
        band[off:, b - off] += -wi - ki
    return band


def random_history(n: int, M: int, seed: int, smooth: bool = False) -> np.ndarray:
    """n x M history block (column-major meaning: column c is one vector of length n)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, M))
    if smooth:
        X = np.cumsum(X, axis=0) / math.sqrt(n)
    return X


def mock_seven_diagonal(n: int, seed: int) -> np.ndarray:
    """Random 7-diagonal matrix with preserved diagonal dominance (the paper's mock test).

    Off-diagonals at offsets -3..3 (excluding 0) ~ U[-1, 1]; a_ii = 1 + sum_j |a_ij|.
    Returned dense (n x n); the right-hand side of that test is u^n = (1, 2, ..., n).
    """
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n))
    for off in (-3, -2, -1, 1, 2, 3):
        vals = rng.uniform(-1.0, 1.0, n)
        for i in range(n):
            j = i + off
            if 0 <= j < n:
                A[i, j] = vals[i]
    A[np.arange(n), np.arange(n)] = 1.0 + np.abs(A).sum(axis=1)
    return A


def dense_to_band(A: np.ndarray, w: int) -> np.ndarray:
    """Row-major band storage band[i, p] = A(i, i + p - w) (zero outside the matrix)."""
    n = A.shape[0]
    band = np.zeros((n, 2 * w + 1))
    for p in range(2 * w + 1):
        off = p - w
        lo, hi = max(0, -off), min(n, n - off)
        band[lo:hi, p] = A[np.arange(lo, hi), np.arange(lo, hi) + off]
    return band


# the sizes of the paper's mock test (Results section)
MOCK_SIZES = (20, 80, 150, 350, 700)
