"""Seeded synthetic inputs for the 1D rotating shallow-water workloads.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no operator, transform, propagator or average).  Both the
CPU oracle (through the tests) and the CUDA path (through the tests and the
bench) take their inputs from here, so the two sides see identical bytes.

Generator (published definitions, written out here):
  * splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
    generators", OOPSLA 2014) produces a 64-bit stream from a 64-bit seed;
  * a uniform in (0, 1) is ((z >> 11) + 0.5) * 2**-53;
  * two uniforms give two independent N(0, 1) variates by the Box-Muller
    transform (Box & Muller 1958).

Spectral layout of a state (shared by every public buffer of the library):
  u[f, k] for field f in (v1, v2, h) and k = 0 .. N/2, complex128, so that the
  physical field is u_f(x_j) = sum_{k=-N/2+1}^{N/2} u[f, k] e^{i k x_j} with
  x_j = 2 pi j / N and u[f, -k] = conj(u[f, k]) (real fields).

The deterministic initial condition of the paper's experiments (Sec. 6.2,
Eq. 6.4) is provided by `paper_initial_state`: its samples on the grid and
their discrete Fourier coefficients, nothing else.

Initial spectra: the drawn values are discrete Fourier coefficients in the
unnormalised convention of FFT libraries, X_k = sum_j u(x_j) e^{-i k x_j}, so
the stored coefficient is u[f, k] = X_k / N.  For 0 < k <= cutoff, Re X_k and
Im X_k are independent N(0, 1/2) (so E|X_k|^2 = 1); X_0 is real N(0, 1); every
bin is multiplied by exp(-k^2 / scale_div); bins above the cutoff are zero.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """The splitmix64 stream: state += golden gamma, then two xor-shift-multiply mixes."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform on the open interval (0, 1) from the top 53 bits."""
        return ((self.next_u64() >> 11) + 0.5) * (2.0 ** -53)

    def normal_pair(self) -> tuple[float, float]:
        """Two independent standard normals by Box-Muller."""
        u1 = self.uniform()
        u2 = self.uniform()
        r = math.sqrt(-2.0 * math.log(u1))
        t = 2.0 * math.pi * u2
        return r * math.cos(t), r * math.sin(t)


def half_bins(n_grid: int) -> int:
    """Number of stored (non-negative) wavenumbers of a real field on N points."""
    return n_grid // 2 + 1


def random_spectrum(n_grid: int, cutoff: int, scale_div: float, seed: int) -> np.ndarray:
    """One seeded initial state u[f, k] = X_k / N, shape (3, N/2+1), complex128.

    Fields are drawn in the order v1, v2, h; within a field, wavenumbers in
    increasing order; each bin consumes one Box-Muller pair.
    """
    if n_grid < 2 or n_grid & (n_grid - 1):
        raise ValueError("grid size must be a power of two")
    h = half_bins(n_grid)
    if cutoff < 0 or cutoff >= h:
        raise ValueError("cutoff must lie in [0, N/2)")
    g = SplitMix64(seed)
    u = np.zeros((3, h), dtype=np.complex128)
    for f in range(3):
        for k in range(cutoff + 1):
            a, b = g.normal_pair()
            amp = math.exp(-(k * k) / scale_div) / n_grid
            if k == 0:
                u[f, 0] = a * amp
            else:
                u[f, k] = complex(a, b) * (amp / math.sqrt(2.0))
    return u


def random_batch(n_grid: int, cutoff: int, scale_div: float, count: int, seed0: int) -> np.ndarray:
    """`count` independent states with seeds seed0, seed0+1, ...; shape (count, 3, N/2+1)."""
    return np.stack([random_spectrum(n_grid, cutoff, scale_div, seed0 + i) for i in range(count)])


@dataclass(frozen=True)
class Workload:
    """One parareal problem: grid, physics, time slicing and quadrature size."""

    name: str
    n_grid: int
    eps: float
    nu: float
    t_end: float
    slices: int
    dt: float
    m_quad: int
    k_max: int
    ic_cutoff: int
    ic_scale_div: float
    seed: int

    @property
    def dT(self) -> float:
        return self.t_end / self.slices

    def initial_state(self) -> np.ndarray:
        return random_spectrum(self.n_grid, self.ic_cutoff, self.ic_scale_div, self.seed)


# The small FP64 parareal problem: N=64, eps=0.01, T=1 over 16 slices,
# fine dt=1e-3, M=32 quadrature points, at most 5 iterations.
SMALL_N64 = Workload("rsw-N64-eps1e-2-S16-M32", 64, 1e-2, 1e-4, 1.0, 16, 1e-3, 32, 5, 8, 16.0, 0)

# The single large instance: N=512, eps=1e-3, T=10 over 256 slices,
# fine dt=1e-4, M=64.
LARGE_N512 = Workload("rsw-N512-eps1e-3-S256-M64", 512, 1e-3, 1e-4, 10.0, 256, 1e-4, 64, 5, 32, 256.0, 0)

# The precision-sweep instance: N=1024, eps=1e-4, T=10 over 512 slices,
# fine dt=1e-5, M=128.
SWEEP_N1024 = Workload("rsw-N1024-eps1e-4-S512-M128", 1024, 1e-4, 1e-4, 10.0, 512, 1e-5, 128, 5, 32, 256.0, 0)


def uneven_instances(count: int, seed: int = 1000):
    """Batched uneven instances: N from {64..1024}, eps log-uniform in [1e-4, 1e-2],
    slices from {32, 64, 128}, M = 32, T = 1, dt = eps/10; instance i uses
    seed `seed + i` for its initial spectrum (cutoff 8, scale e^{-k^2/16})."""
    g = SplitMix64(seed ^ 0x5EED)
    out = []
    for i in range(count):
        n_grid = (64, 128, 256, 512, 1024)[g.next_u64() % 5]
        eps = 10.0 ** (-4.0 + 2.0 * g.uniform())
        slices = (32, 64, 128)[g.next_u64() % 3]
        out.append(Workload(f"uneven-{i}", n_grid, eps, 1e-4, 1.0, slices, eps / 10.0, 32, 5, 8, 16.0, seed + i))
    return out


def paper_height_profile(x: np.ndarray) -> np.ndarray:
    """The bracket of Eq. 6.4 (Sec. 6.2): two Gaussian-windowed sines."""
    a = x - math.pi / 2.0
    b = x - math.pi
    return np.exp(-4.0 * a * a) * np.sin(3.0 * a) + np.exp(-2.0 * b * b) * np.sin(8.0 * b)


def paper_height_constants(fine: int = 1 << 16) -> tuple[float, float]:
    """c1, c0 of Eq. 6.4: h = c1 f + c0 with zero mean over [0, 2 pi) and
    max |h| = 1, both evaluated on `fine` equispaced points."""
    x = 2.0 * math.pi * np.arange(fine) / fine
    f = paper_height_profile(x)
    mean = float(np.mean(f))
    c1 = 1.0 / float(np.max(np.abs(f - mean)))
    return c1, -c1 * mean


def paper_initial_state(n_grid: int) -> np.ndarray:
    """Sec. 6.2's initial condition on N points: v1 = v2 = 0 and h of Eq. 6.4,
    stored as u[2, k] = X_k / N from the samples h(x_j), shape (3, N/2+1)."""
    if n_grid < 2 or n_grid & (n_grid - 1):
        raise ValueError("grid size must be a power of two")
    c1, c0 = paper_height_constants()
    x = 2.0 * math.pi * np.arange(n_grid) / n_grid
    h = c1 * paper_height_profile(x) + c0
    u = np.zeros((3, half_bins(n_grid)), dtype=np.complex128)
    u[2] = np.fft.rfft(h) / n_grid
    return u


@dataclass(frozen=True)
class PaperExperiment:
    """One experiment of Sec. 6.2: the asymptotic method's dT, dt, fast-time
    averaging window T0 and M (nodes), its number of slices, and the coarse steps of the
    standard-parareal comparison runs (Strang coarse solver, same dt, same
    horizon).  Grid, horizons and the conflicting printed values are readings
    (see the experiment tables)."""
    name: str
    eps: float
    dT: float
    dt: float
    window: float
    m_quad: int
    slices: int
    standard_dT: tuple
    n_grid: int = 128
    nu: float = 1e-4

    @property
    def t_end(self) -> float:
        return self.slices * self.dT


# eps = 1e-2: dT = 50 eps, dt = eps/25, averaging over 150 eps of physical
# time, M = 450; standard parareal with dT = 4 eps and 5 eps.  eps = 1e-1:
# dT = 3 eps, dt = eps/50, 5 eps of physical time, M = 10, 150 slices; standard
# with dT = eps and 2 eps.  eps = 1: dT = 3/10, dt = 1/200, 3/10 of physical
# time, M = 10, 60 slices; standard with dT = 3/10 and 4/10.  `window` is the
# fast-time window (the physical one divided by eps).
PAPER_EXPERIMENTS = (
    PaperExperiment("paper-eps1e-2", 1e-2, 0.5, 1e-2 / 25, 150.0, 450, 128, (0.04, 0.05)),
    PaperExperiment("paper-eps1e-1", 1e-1, 0.3, 1e-1 / 50, 5.0, 10, 150, (0.1, 0.2)),
    PaperExperiment("paper-eps1", 1.0, 0.3, 1.0 / 200, 0.3, 10, 60, (0.3, 0.4)),
)
