"""FP64 oracle: what the asymptotic parareal hot path computes, written plainly.

TEST INFRASTRUCTURE ONLY (tests/, __graft_entry__.smoke(), bench.py's CPU
baseline).  Slow and direct on purpose; it shares no code with the CUDA path.

Model (Haut & Wingate, Sec. 6.1, Eq. 6.1): u = (v1, v2, h) on the periodic
interval [0, 2 pi), written in the generic form of Eq. 1.1,

    du/dt + (1/eps) L u = N(u) + D u,

with, in Fourier space (d/dx -> i k, F = 1 unless set otherwise):

    L_k = [[0, -1, i k F^-1/2], [1, 0, 0], [i k F^-1/2, 0, 0]]   (Sec. 6.1)
    D_k = -nu k^4                 (reading: the printed +mu d^4/dx^4 is meant
                                   as dissipation, so its symbol is -nu k^4)
    N(u) = -(v1 v1_x, v1 v2_x, (h v1)_x)   (reading: signs of the explicit
                                   PDE of Eq. 6.1, advection on the left side)

State layout: complex128 arrays (..., 3, N/2+1) of the Fourier coefficients
u[f, k] of the real fields, u_f(x_j) = sum_k u[f, k] e^{i k x_j}, x_j = 2 pi j/N.
Every routine works in this physical spectral basis; the stiff linear part is
applied as a 3x3 matrix function per wavenumber, obtained from the Hermitian
eigendecomposition of -i L_k (so L_k = V diag(i omega) V^H, Sec. 6.1).

Dealiasing (the paper is silent): the 2/3 rule, keeping |k| <= K = floor((N-1)/3),
so quadratic products of kept modes are formed without aliasing (3K < N).
The state space is the kept band with real k = 0 coefficients; `project`
maps any input onto it (bins above K and Im of the k = 0 bins are dropped).

Functions and the passages they follow:
  nonlinear            N(u) by transform, product, dealias (Sec. 6.1 operator table)
  etdrk4_coefficients  Cox & Matthews ETDRK4 weights (named in Sec. 6.2; ref. [CoxMathews])
  fine_step/fine_propagate   the fine propagator phi_dT (Sec. 3 notation; Sec. 6.2 uses ETDRK4)
  rho, quadrature      kernel and nodes of Eq. 2.1-2.2 and Algorithm 1
  nbar                 finite, discretised average of Eq. 2.1 (Algorithm 1)
  coarse_step          asymptotic slow solver (Algorithm 2)
  strang_step/strang_propagate   Strang-splitting fine solver (Algorithm 3)
  ifrk4_step/ifrk4_propagate     integrating-factor RK4, the comparator of Sec. 6.2
                       (the integrating factor method of Kassam & Trefethen)
  coarse_step_strang   one Strang step over dT: the coarse solver of standard
                       parareal on the full equation (Sec. 6.2)
  restrict_state/prolong_state/coarse_step_on_grid   the asymptotic solver on a
                       coarser grid (the remark on a coarser spatial discretisation, Sec. 1)
  parareal             the iteration of Eq. 3.1 (Algorithm 4)
  rel_change_norm      stopping quantity of Algorithm 4
  estimated_speedup    complexity model of Eq. 5.1

Readings where the paper is silent or inconsistent (each also used by the CUDA
path, and listed with reasons in the design notes):
  * s in e^{sL} is fast time; the window T0 is in fast-time units (Sec. 2 uses
    both e^{sL} and e^{(s/eps)L}); default T0 = dT/eps (the eps = O(1) rule of
    Sec. 4, one coarse step).
  * nodes s_m = T0 m / M, m = 0..M-1, weights rho(m/M)/M with the literal
    normalisation int_0^1 rho = 1 (Algorithm 1 / Eq. 2.2).
  * Algorithm 2's last factor is e^{-(dT/eps) L} (the map back to fast time of
    Sec. 3, u = e^{-t L/eps} u_bar), and its two N_bar evaluations form the
    explicit midpoint rule on the half-D-stepped state.
  * fine steps per slice = ceil(dT/dt - 1e-9), h = dT / steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np
from scipy import integrate

__all__ = [
    "kept_modes", "half_bins", "Params", "fine_steps", "L_symbol", "L_eigen",
    "project", "synthesize", "analyze", "nonlinear", "linear_matrices",
    "phi123", "etdrk4_coefficients", "fine_step", "fine_propagate",
    "bump_integral", "rho", "quadrature", "expL", "nbar", "coarse_step",
    "parareal", "serial_fine", "parseval_norm", "rel_change_norm",
    "physical_linf", "estimated_speedup",
]


# ---------------------------------------------------------------------------
# layout
# ---------------------------------------------------------------------------

def kept_modes(n_grid: int) -> int:
    """Largest kept wavenumber K under the 2/3 rule (3K < N)."""
    return (n_grid - 1) // 3


def half_bins(n_grid: int) -> int:
    return n_grid // 2 + 1


@dataclass
class Params:
    """One problem: grid N, Rossby number eps, hyperviscosity nu, coarse step
    dT, fine step dt, quadrature size M, window T0 (fast time; None -> dT/eps)
    and the free parameter F of Eq. 6.1 (set to 1 in Sec. 6.1)."""

    n_grid: int
    eps: float
    nu: float
    dT: float
    dt: float
    m_quad: int
    T0: Optional[float] = None
    F: float = 1.0
    _cache: dict = field(default_factory=dict, repr=False, compare=False)

    @property
    def K(self) -> int:
        return kept_modes(self.n_grid)

    @property
    def H(self) -> int:
        return half_bins(self.n_grid)

    @property
    def window(self) -> float:
        return self.dT / self.eps if self.T0 is None else self.T0


def fine_steps(dT: float, dt: float) -> tuple[int, float]:
    """Fine steps per slice and their size (dt need not divide dT)."""
    steps = int(math.ceil(dT / dt - 1e-9))
    steps = max(steps, 1)
    return steps, dT / steps


# ---------------------------------------------------------------------------
# linear operator (Sec. 6.1)
# ---------------------------------------------------------------------------

def L_symbol(k: float, F: float = 1.0) -> np.ndarray:
    """Fourier symbol of L at wavenumber k (d/dx -> i k)."""
    g = 1j * k / math.sqrt(F)
    return np.array([[0.0, -1.0, g], [1.0, 0.0, 0.0], [g, 0.0, 0.0]], dtype=np.complex128)


def L_eigen(k: float, F: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """omega (ascending) and unitary V with L_k V = V diag(i omega).

    -i L_k is Hermitian because L_k is skew-Hermitian, so numpy's Hermitian
    eigensolver gives real omega and orthonormal eigenvectors."""
    w, V = np.linalg.eigh(-1j * L_symbol(k, F))
    return w, V


def _eigen_table(p: Params):
    key = ("eig", p.n_grid, p.F)
    if key not in p._cache:
        ks = np.arange(p.H)
        om = np.zeros((p.H, 3))
        V = np.zeros((p.H, 3, 3), dtype=np.complex128)
        for k in ks:
            om[k], V[k] = L_eigen(float(k), p.F)
        p._cache[key] = (om, V)
    return p._cache[key]


def _matfun(p: Params, fvals: np.ndarray) -> np.ndarray:
    """Per-k matrices V diag(fvals[k]) V^H, shape (H, 3, 3)."""
    _, V = _eigen_table(p)
    return np.einsum("kia,ka,kja->kij", V, fvals, V.conj())


def _apply(mats: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Apply per-k 3x3 matrices (H,3,3) to states (...,3,H)."""
    return np.einsum("kij,...jk->...ik", mats, u)


# ---------------------------------------------------------------------------
# spectral <-> physical, projection, nonlinearity (Sec. 6.1)
# ---------------------------------------------------------------------------

def project(u: np.ndarray, n_grid: int) -> np.ndarray:
    """Map onto the state space: bins k > K set to zero, k = 0 bins made real."""
    K = kept_modes(n_grid)
    out = np.array(u, dtype=np.complex128, copy=True)
    out[..., K + 1:] = 0.0
    out[..., 0] = out[..., 0].real
    return out


def synthesize(uh: np.ndarray, n_grid: int) -> np.ndarray:
    """Physical samples u(x_j) = sum_k uh_k e^{i k x_j} of real fields."""
    return np.fft.irfft(uh, n=n_grid, axis=-1) * n_grid


def analyze(x: np.ndarray, n_grid: int) -> np.ndarray:
    """Coefficients uh_k = (1/N) sum_j x_j e^{-i k x_j}, k = 0..N/2."""
    return np.fft.rfft(x, n=n_grid, axis=-1) / n_grid


def nonlinear(u: np.ndarray, n_grid: int) -> np.ndarray:
    """N(u) = -(v1 v1_x, v1 v2_x, (h v1)_x), pseudo-spectrally with the 2/3 rule."""
    K = kept_modes(n_grid)
    ik = 1j * np.arange(half_bins(n_grid))
    u = project(u, n_grid)
    v1 = synthesize(u[..., 0, :], n_grid)
    v1x = synthesize(ik * u[..., 0, :], n_grid)
    v2x = synthesize(ik * u[..., 1, :], n_grid)
    h = synthesize(u[..., 2, :], n_grid)
    out = np.empty_like(u)
    out[..., 0, :] = -analyze(v1 * v1x, n_grid)
    out[..., 1, :] = -analyze(v1 * v2x, n_grid)
    out[..., 2, :] = -ik * analyze(h * v1, n_grid)
    out[..., K + 1:] = 0.0
    return out


# ---------------------------------------------------------------------------
# ETDRK4 (Cox & Matthews 2002), the fine propagator
# ---------------------------------------------------------------------------

def phi123(z: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """phi_j(z) = sum_{n>=0} z^n/(n+j)!, j = 1, 2, 3.

    Power series where |z| < 1 (30 terms; the tail is below 1e-30 there);
    elsewhere the closed forms (e^z - 1)/z, (e^z - 1 - z)/z^2,
    (e^z - 1 - z - z^2/2)/z^3."""
    z = np.asarray(z, dtype=np.complex128)
    p1 = np.empty_like(z)
    p2 = np.empty_like(z)
    p3 = np.empty_like(z)
    small = np.abs(z) < 1.0
    zs = z[small]
    s1 = np.zeros_like(zs)
    s2 = np.zeros_like(zs)
    s3 = np.zeros_like(zs)
    term = np.ones_like(zs)  # z^n
    for n in range(30):
        s1 += term / math.factorial(n + 1)
        s2 += term / math.factorial(n + 2)
        s3 += term / math.factorial(n + 3)
        term = term * zs
    p1[small], p2[small], p3[small] = s1, s2, s3
    zb = z[~small]
    ez = np.exp(zb)
    p1[~small] = (ez - 1.0) / zb
    p2[~small] = (ez - 1.0 - zb) / zb**2
    p3[~small] = (ez - 1.0 - zb - zb**2 / 2.0) / zb**3
    return p1, p2, p3


def linear_eigenvalues(p: Params) -> np.ndarray:
    """lambda = -i omega/eps - nu k^4 per (k, eigen-branch), shape (H, 3).
    eps = inf switches the fast term off."""
    om, _ = _eigen_table(p)
    k4 = (np.arange(p.H, dtype=np.float64) ** 4)[:, None]
    fast = np.zeros_like(om) if math.isinf(p.eps) else om / p.eps
    return -1j * fast - p.nu * k4


def linear_matrices(p: Params, t: float) -> np.ndarray:
    """e^{t (-L/eps + D)} per k, shape (H, 3, 3)."""
    return _matfun(p, np.exp(t * linear_eigenvalues(p)))


def etdrk4_coefficients(p: Params, h: float) -> dict:
    """Per-k 3x3 matrices of one ETDRK4 step of size h for u' = A u + N(u):
    E = e^{hA}, E2 = e^{hA/2}, Q = (h/2) phi1(hA/2),
    f1 = h(phi1 - 3 phi2 + 4 phi3)(hA), f2 = h(phi2 - 2 phi3)(hA),
    f3 = h(4 phi3 - phi2)(hA)."""
    key = ("etd", h, p.eps, p.nu, p.n_grid, p.F)
    if key in p._cache:
        return p._cache[key]
    lam = linear_eigenvalues(p)
    z = h * lam
    a1, a2, a3 = phi123(z)
    b1, _, _ = phi123(z / 2.0)
    c = {
        "E": _matfun(p, np.exp(z)),
        "E2": _matfun(p, np.exp(z / 2.0)),
        "Q": _matfun(p, (h / 2.0) * b1),
        "f1": _matfun(p, h * (a1 - 3.0 * a2 + 4.0 * a3)),
        "f2": _matfun(p, h * (a2 - 2.0 * a3)),
        "f3": _matfun(p, h * (4.0 * a3 - a2)),
    }
    p._cache[key] = c
    return c


NonlinearFn = Callable[[np.ndarray, int], np.ndarray]


def fine_step(u: np.ndarray, p: Params, h: float, nl: NonlinearFn = nonlinear) -> np.ndarray:
    """One ETDRK4 step (Cox & Matthews):
        a = E2 u + Q N(u)
        b = E2 u + Q N(a)
        c = E2 a + Q (2 N(b) - N(u))
        u+ = E u + f1 N(u) + 2 f2 (N(a) + N(b)) + f3 N(c)."""
    c = etdrk4_coefficients(p, h)
    n = p.n_grid
    Nu = nl(u, n)
    a = _apply(c["E2"], u) + _apply(c["Q"], Nu)
    Na = nl(a, n)
    b = _apply(c["E2"], u) + _apply(c["Q"], Na)
    Nb = nl(b, n)
    cc = _apply(c["E2"], a) + _apply(c["Q"], 2.0 * Nb - Nu)
    Nc = nl(cc, n)
    return (_apply(c["E"], u) + _apply(c["f1"], Nu) + 2.0 * _apply(c["f2"], Na + Nb)
            + _apply(c["f3"], Nc))


def fine_propagate(u: np.ndarray, p: Params, nl: NonlinearFn = nonlinear,
                   steps: Optional[int] = None) -> np.ndarray:
    """The fine propagator over one coarse interval dT: `steps` ETDRK4 steps."""
    if steps is None:
        steps, h = fine_steps(p.dT, p.dt)
    else:
        h = p.dT / steps
    u = project(u, p.n_grid)
    for _ in range(steps):
        u = fine_step(u, p, h, nl)
    return u


# ---------------------------------------------------------------------------
# Strang splitting (Algorithm 3) and standard parareal's coarse solver (Sec. 6.2)
# ---------------------------------------------------------------------------

def _linear_half(p: Params, h: float) -> np.ndarray:
    key = ("lin_half", h, p.eps, p.nu, p.n_grid, p.F)
    if key not in p._cache:
        p._cache[key] = linear_matrices(p, h / 2.0)
    return p._cache[key]


def strang_step(u: np.ndarray, p: Params, h: float, nl: NonlinearFn = nonlinear) -> np.ndarray:
    """One Strang-splitting step of size h (Algorithm 3): an exact half step of
    the linear part, a midpoint step of the nonlinear part, an exact half step.
    The nonlinear stage is read as in Algorithm 2:
        w = e^{h/2 (-L/eps + D)} u;  k1 = N(w);  k2 = N(w + h/2 k1);  w = w + h k2;
        return e^{h/2 (-L/eps + D)} w."""
    E2 = _linear_half(p, h)
    n = p.n_grid
    w = _apply(E2, u)
    k1 = nl(w, n)
    k2 = nl(w + (h / 2.0) * k1, n)
    w = w + h * k2
    return _apply(E2, w)


def strang_propagate(u: np.ndarray, p: Params, nl: NonlinearFn = nonlinear,
                     steps: Optional[int] = None) -> np.ndarray:
    """The Strang-splitting fine propagator over one coarse interval dT."""
    if steps is None:
        steps, h = fine_steps(p.dT, p.dt)
    else:
        h = p.dT / steps
    u = project(u, p.n_grid)
    for _ in range(steps):
        u = strang_step(u, p, h, nl)
    return u


def ifrk4_step(u: np.ndarray, p: Params, h: float, nl: NonlinearFn = nonlinear) -> np.ndarray:
    """One integrating-factor RK4 step: classical RK4 applied to
    v = e^{-t A} u, A = -L/eps + D, so that v' = e^{-t A} N(e^{t A} v), mapped
    back (E = e^{hA}, E2 = e^{hA/2}):
        k1 = N(u);  k2 = N(E2 (u + h/2 k1));  k3 = N(E2 u + h/2 k2);
        k4 = N(E u + h E2 k3);
        u+ = E u + h/6 (E k1 + 2 E2 (k2 + k3) + k4)."""
    E2 = _linear_half(p, h)
    E = _linear_half(p, 2.0 * h)
    n = p.n_grid
    k1 = nl(u, n)
    k2 = nl(_apply(E2, u + (h / 2.0) * k1), n)
    k3 = nl(_apply(E2, u) + (h / 2.0) * k2, n)
    k4 = nl(_apply(E, u) + h * _apply(E2, k3), n)
    return _apply(E, u) + (h / 6.0) * (_apply(E, k1) + 2.0 * _apply(E2, k2 + k3) + k4)


def ifrk4_propagate(u: np.ndarray, p: Params, nl: NonlinearFn = nonlinear,
                    steps: Optional[int] = None) -> np.ndarray:
    """The integrating-factor RK4 fine propagator over one coarse interval dT."""
    if steps is None:
        steps, h = fine_steps(p.dT, p.dt)
    else:
        h = p.dT / steps
    u = project(u, p.n_grid)
    for _ in range(steps):
        u = ifrk4_step(u, p, h, nl)
    return u


def coarse_step_strang(u: np.ndarray, p: Params, nl: NonlinearFn = nonlinear) -> np.ndarray:
    """Standard parareal's coarse solver (Sec. 6.2): one Strang step of size dT
    of the full equation."""
    return strang_step(project(u, p.n_grid), p, p.dT, nl)


# ---------------------------------------------------------------------------
# time average (Sec. 2, Eq. 2.1-2.2, Algorithm 1) and the slow solver (Algorithm 2)
# ---------------------------------------------------------------------------

def bump_integral() -> float:
    """int_0^1 exp(-1/(s(1-s))) ds (so the kernel's constant is its inverse)."""
    val, _ = integrate.quad(lambda s: math.exp(-1.0 / (s * (1.0 - s))), 0.0, 1.0,
                            epsabs=1e-17, epsrel=1e-13, limit=200)
    return val


_BUMP = None


def rho(s: np.ndarray) -> np.ndarray:
    """rho(s) = C exp(-1/(s(1-s))) on (0,1), 0 elsewhere, with int rho = 1 (Sec. 2)."""
    global _BUMP
    if _BUMP is None:
        _BUMP = bump_integral()
    s = np.asarray(s, dtype=np.float64)
    out = np.zeros_like(s)
    inside = (s > 0.0) & (s < 1.0)
    si = s[inside]
    out[inside] = np.exp(-1.0 / (si * (1.0 - si))) / _BUMP
    return out


def quadrature(p: Params) -> tuple[np.ndarray, np.ndarray]:
    """Nodes s_m = T0 m/M (fast time) and weights rho(m/M)/M, m = 0..M-1."""
    m = np.arange(p.m_quad, dtype=np.float64)
    return p.window * m / p.m_quad, rho(m / p.m_quad) / p.m_quad


def expL(p: Params, s: float) -> np.ndarray:
    """e^{s L} per k (unitary), shape (H, 3, 3)."""
    om, _ = _eigen_table(p)
    return _matfun(p, np.exp(1j * s * om))


def nbar(u: np.ndarray, p: Params, nl: NonlinearFn = nonlinear) -> np.ndarray:
    """Averaged nonlinearity: sum_m w_m e^{s_m L} N(e^{-s_m L} u)  (Eq. 2.1 / Algorithm 1)."""
    s, w = quadrature(p)
    u = project(u, p.n_grid)
    acc = np.zeros_like(u)
    for sm, wm in zip(s, w):
        acc = acc + wm * _apply(expL(p, sm), nl(_apply(expL(p, -sm), u), p.n_grid))
    return acc


def coarse_step(u: np.ndarray, p: Params, nl: NonlinearFn = nonlinear) -> np.ndarray:
    """Asymptotic slow solver over dT (Algorithm 2):
        w = e^{dT/2 D} u;  k1 = Nbar(w);  k2 = Nbar(w + dT/2 k1);  w = w + dT k2;
        w = e^{dT/2 D} w;  return e^{-(dT/eps) L} w."""
    dT = p.dT
    k4 = np.arange(p.H, dtype=np.float64) ** 4
    dhalf = np.exp(-p.nu * k4 * dT / 2.0)
    w = dhalf * project(u, p.n_grid)
    k1 = nbar(w, p, nl)
    k2 = nbar(w + (dT / 2.0) * k1, p, nl)
    w = w + dT * k2
    w = dhalf * w
    fast = 0.0 if math.isinf(p.eps) else dT / p.eps
    return _apply(expL(p, -fast), w)


def restrict_state(u: np.ndarray, n_coarse: int) -> np.ndarray:
    """The modes of u representable on n_coarse points, projected there (k <= K_c)."""
    return project(np.array(u[..., : half_bins(n_coarse)], copy=True), n_coarse)


def prolong_state(v: np.ndarray, n_grid: int) -> np.ndarray:
    """A coarse-grid state on n_grid points: the missing modes are zero."""
    out = np.zeros(v.shape[:-1] + (half_bins(n_grid),), dtype=np.complex128)
    out[..., : v.shape[-1]] = v
    return out


def coarse_step_on_grid(u: np.ndarray, p: Params, n_coarse: int, nl: NonlinearFn = nonlinear) -> np.ndarray:
    """The asymptotic slow solver (Algorithm 2) run on n_coarse points: restrict,
    step with the same eps, nu, dT, window and nodes, prolong."""
    pc = Params(n_coarse, p.eps, p.nu, p.dT, p.dt, p.m_quad, T0=p.T0, F=p.F)
    return prolong_state(coarse_step(restrict_state(u, n_coarse), pc, nl), p.n_grid)


# ---------------------------------------------------------------------------
# parareal (Sec. 3, Eq. 3.1, Algorithm 4)
# ---------------------------------------------------------------------------

def parseval_norm(u: np.ndarray) -> np.ndarray:
    """L2 norm over the three fields via Parseval (weight 1 at k=0, 2 above);
    the Nyquist bin is zero in the state space.  Reduces the last two axes."""
    wgt = np.full(u.shape[-1], 2.0)
    wgt[0] = 1.0
    return np.sqrt(np.sum(wgt * np.abs(u) ** 2, axis=(-2, -1)))


def rel_change_norm(new: np.ndarray, old: np.ndarray) -> float:
    """max_n ||new_n - old_n|| / ||new_n|| over slices n (Algorithm 4's stopping
    quantity); a slice whose new norm is zero counts 0 if unchanged, else inf."""
    d = parseval_norm(new - old)
    nn = parseval_norm(new)
    r = np.where(nn > 0, d / np.where(nn > 0, nn, 1.0), np.where(d > 0, np.inf, 0.0))
    return float(np.max(r))


@dataclass
class PararealResult:
    iterates: list          # U^k for k = 0..k_done, each (S+1, 3, H)
    changes: list           # max relative change after each k >= 1


def parareal(u0: np.ndarray, p: Params, slices: int, k_max: int, tol: float = 0.0,
             F: Optional[Callable] = None, G: Optional[Callable] = None) -> PararealResult:
    """U_0^k = u0; U_n^0 = G(U_{n-1}^0);
    U_n^k = G(U_{n-1}^k) + F(U_{n-1}^{k-1}) - G(U_{n-1}^{k-1})  (Eq. 3.1),
    stopping after k_max iterations or once the relative change is <= tol."""
    F = F or (lambda x: fine_propagate(x, p))
    G = G or (lambda x: coarse_step(x, p))
    u0 = project(u0, p.n_grid)
    U = [u0]
    for n in range(1, slices + 1):
        U.append(G(U[n - 1]))
    U = np.stack(U)
    res = PararealResult([U], [])
    for _ in range(k_max):
        f_old = F(U[:-1])
        g_old = G(U[:-1])
        new = [u0]
        for n in range(1, slices + 1):
            new.append(G(new[n - 1]) + f_old[n - 1] - g_old[n - 1])
        new = np.stack(new)
        ch = rel_change_norm(new[1:], U[1:])
        U = new
        res.iterates.append(U)
        res.changes.append(ch)
        if ch <= tol:
            break
    return res


def serial_fine(u0: np.ndarray, p: Params, slices: int) -> np.ndarray:
    """u(n dT) ~ F^n(u0), n = 0..slices: what parareal converges to."""
    out = [project(u0, p.n_grid)]
    for _ in range(slices):
        out.append(fine_propagate(out[-1], p))
    return np.stack(out)


def physical_linf(u: np.ndarray, n_grid: int) -> np.ndarray:
    """max over grid points and fields of |u_f(x_j)|; reduces the last two axes."""
    return np.max(np.abs(synthesize(u, n_grid)), axis=(-2, -1))


def estimated_speedup(n_slices: float, m_ratio: float, iters: float,
                      tau_f: float = 1.0, tau_c: float = 1.0) -> float:
    """Eq. 5.1: tau_f N M / (nu (tau_f M + tau_c N + tau_c) + tau_c N), with N
    slices, M = dT/dt fine steps per slice and nu iterations."""
    return tau_f * n_slices * m_ratio / (iters * (tau_f * m_ratio + tau_c * n_slices + tau_c)
                                         + tau_c * n_slices)
