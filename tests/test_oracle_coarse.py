"""Oracle pins for the averaged nonlinearity (Eq. 2.1-2.2, Algorithm 1, Eq. 6.2)
and the asymptotic slow solver (Algorithm 2)."""
import math

import mpmath
import numpy as np
import pytest
from scipy.linalg import expm

import rsw_inputs as ri
from oracle import rsw as o


def test_kernel_normalisation_constant():
    # rho = C exp(-1/(s(1-s))) with ||rho||_1 = 1 (Sec. 2); C from 40-digit quadrature.
    mpmath.mp.dps = 40
    ref = mpmath.quad(lambda s: mpmath.exp(-1 / (s * (1 - s))), [0, 0.5, 1])
    assert abs(o.bump_integral() / float(ref) - 1) < 1e-13
    assert abs(1 / float(ref) - 142.25037577709588) < 1e-11
    # the kernel and all its derivatives vanish at the ends; it peaks at s = 1/2
    assert o.rho(np.array([0.0, 1.0, -0.2, 1.3])).tolist() == [0.0, 0.0, 0.0, 0.0]
    assert abs(o.rho(np.array([0.5]))[0] - math.exp(-4) / float(ref)) < 1e-12


@pytest.mark.parametrize("m", [10, 32, 64, 128])
def test_quadrature_weights_sum_to_one(m):
    # trapezoid rule on a flat-ended kernel: sum of weights -> int rho = 1 super-algebraically
    p = o.Params(16, 0.01, 0.0, 0.1, 0.01, m, T0=7.0)
    s, w = o.quadrature(p)
    np.testing.assert_allclose(s, 7.0 * np.arange(m) / m)
    assert w[0] == 0.0
    tol = {10: 5e-4, 32: 1e-7, 64: 1e-11, 128: 1e-14}[m]
    assert abs(w.sum() - 1.0) < tol


def _closed_form_eigvecs(k):
    """Columns r^{-1}, r^0, r^{+1} of Sec. 6.1 in closed form (F = 1)."""
    sg = math.sqrt(1 + k * k)
    rm = np.array([1, 1j / sg, -k / sg]) / math.sqrt(2)
    r0 = np.array([0, 1j * k, 1]) / sg
    rp = np.array([1, -1j / sg, k / sg]) / math.sqrt(2)
    return np.stack([rm, r0, rp], axis=1), np.array([-sg, 0.0, sg])


def _triad_nbar(u, n, W):
    """Eq. 6.2 summed directly: for each k and branch alpha,
    sum_{k1+k2=k} sum_{a1,a2} W(omega - omega1 - omega2) C u^{a1}_{k1} u^{a2}_{k2},
    with C = r_k^H B(r_{k1} e^{ik1x}, r_{k2} e^{ik2x}) and
    B(u, w) = -(u1 w1_x, u1 w2_x, (u1 w3)_x), so that N(u) = B(u, u)."""
    K = o.kept_modes(n)

    def full(k):
        return u[:, k] if k >= 0 else np.conj(u[:, -k])

    eig = {k: _closed_form_eigvecs(k) for k in range(-K, K + 1)}
    amp = {k: eig[k][0].conj().T @ full(k) for k in range(-K, K + 1)}
    out = np.zeros((3, n // 2 + 1), dtype=complex)
    for k in range(0, K + 1):
        R, om = eig[k]
        acc = np.zeros(3, dtype=complex)
        for k1 in range(-K, K + 1):
            k2 = k - k1
            if abs(k2) > K:
                continue
            R1, om1 = eig[k1]
            R2, om2 = eig[k2]
            for a1 in range(3):
                for a2 in range(3):
                    r1, r2 = R1[:, a1], R2[:, a2]
                    B = -np.array([r1[0] * 1j * k2 * r2[0], r1[0] * 1j * k2 * r2[1],
                                   1j * k * r1[0] * r2[2]])
                    coef = R.conj().T @ B       # C for the three output branches
                    for a in range(3):
                        acc[a] += W(om[a] - om1[a1] - om2[a2]) * coef[a] * amp[k1][a1] * amp[k2][a2]
        out[:, k] = R @ acc
    return out


def _quadrature_filter(s_nodes, w):
    """W(d) = sum_m w_m e^{i d s_m}."""
    return lambda d: np.sum(w * np.exp(1j * d * s_nodes))


@pytest.mark.parametrize("n,m,T0", [(8, 6, 3.0), (16, 12, 9.5)])
def test_nbar_equals_brute_force_triad_sum(n, m, T0):
    p = o.Params(n, 0.01, 0.0, 0.1, 0.01, m, T0=T0)
    rng = np.random.default_rng(n + m)
    K = o.kept_modes(n)
    u = np.zeros((3, n // 2 + 1), dtype=complex)
    u[:, :K + 1] = rng.standard_normal((3, K + 1)) + 1j * rng.standard_normal((3, K + 1))
    u[:, 0] = u[:, 0].real
    s, w = o.quadrature(p)
    got = o.nbar(u, p)
    ref = _triad_nbar(u, n, _quadrature_filter(s, w))
    np.testing.assert_allclose(got, ref, atol=1e-13 * np.max(np.abs(ref)))


def _geostrophic_state(n, seed):
    """Only omega = 0 components: u_k = a_k (0, ik, 1)/sqrt(1+k^2), so v1 = 0."""
    rng = np.random.default_rng(seed)
    K = o.kept_modes(n)
    u = np.zeros((3, n // 2 + 1), dtype=complex)
    for k in range(K + 1):
        a = rng.standard_normal() + (1j * rng.standard_normal() if k else 0)
        u[:, k] = a * np.array([0, 1j * k, 1]) / math.sqrt(1 + k * k)
    return u


def test_geostrophic_state_only_decays():
    # Slow modes have v1 = 0, so N = 0 and every propagator reduces to e^{-nu k^4 t}.
    p = o.Params(32, 0.01, 1e-3, 0.0625, 1e-3, 16)
    u0 = _geostrophic_state(32, 4)
    decay = np.exp(-p.nu * np.arange(p.H) ** 4 * p.dT)
    np.testing.assert_allclose(o.fine_propagate(u0, p), decay * u0, atol=1e-13)
    np.testing.assert_allclose(o.coarse_step(u0, p), decay * u0, atol=1e-13)
    np.testing.assert_allclose(o.nbar(u0, p), 0 * u0, atol=1e-14)


def test_coarse_step_linear_part_exact():
    # Nbar off: G(u) = e^{-(dT/eps) L} e^{dT D} u, here via scipy's matrix exponential.
    p = o.Params(32, 0.01, 1e-3, 0.0625, 1e-3, 16)
    u0 = ri.random_spectrum(32, 8, 16.0, 3)
    zero = lambda u, n: np.zeros_like(u)
    got = o.coarse_step(u0, p, nl=zero)
    for k in range(p.H):
        M = expm(-(p.dT / p.eps) * o.L_symbol(float(k))) * math.exp(-p.nu * k ** 4 * p.dT)
        np.testing.assert_allclose(got[:, k], M @ o.project(u0, 32)[:, k], atol=1e-15)


def test_coarse_step_is_second_order():
    # Algorithm 2 (midpoint on Nbar between exact half steps of D, then the exact fast
    # phase) has local error O(dT^3) against the averaged ODE v' = Nbar(v) + D v at
    # fixed window and nodes; reference: classical RK4 with 64 substeps (test-local).
    n = 16
    u0 = 40.0 * ri.random_spectrum(n, 5, 16.0, 8)
    errs = []
    for dT in (0.04, 0.02, 0.01):
        p = o.Params(n, 0.05, 2e-3, dT, dT, 12, T0=4.0)
        k4 = np.arange(p.H) ** 4
        rhs = lambda v: o.nbar(v, p) - p.nu * k4 * v
        v = o.project(u0, n)
        hh = dT / 64
        for _ in range(64):
            a = rhs(v)
            b = rhs(v + hh / 2 * a)
            c = rhs(v + hh / 2 * b)
            d = rhs(v + hh * c)
            v = v + hh / 6 * (a + 2 * b + 2 * c + d)
        ref = np.stack([expm(-(dT / p.eps) * o.L_symbol(float(k))) @ v[:, k] for k in range(p.H)], axis=1)
        errs.append(o.parseval_norm(o.coarse_step(u0, p) - ref))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(r > 6.0 for r in ratios), (errs, ratios)


def test_nbar_approaches_resonant_average_with_long_windows():
    # As T0 grows (and M with it) the filter W(d) -> [d == 0]: Nbar tends to the
    # resonant-set sum of Eq. 6.3.  Checked as a trend on a tiny grid.
    n = 8
    rng = np.random.default_rng(11)
    u = np.zeros((3, 5), dtype=complex)
    u[:, :3] = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    u[:, 0] = u[:, 0].real
    exact = _triad_nbar(u, n, lambda d: 1.0 if abs(d) < 1e-9 else 0.0)
    errs = []
    for T0, m in ((20.0, 64), (80.0, 256), (320.0, 1024)):
        p = o.Params(n, 0.01, 0.0, 0.1, 0.01, m, T0=T0)
        errs.append(o.parseval_norm(o.nbar(u, p) - exact))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.05 * o.parseval_norm(exact)


def test_time_average_on_a_coarser_grid():
    # For a state whose modes all fit the coarse grid's kept band, the 2/3 rule
    # makes every product exact on both grids: the coarse-grid average equals the
    # fine-grid average restricted to the coarse band (and G on the fine grid is
    # G on a "coarse" grid of the same size).
    n, nc = 64, 32
    p = o.Params(n, 0.01, 1e-4, 0.0625, 1e-3, 16)
    pc = o.Params(nc, 0.01, 1e-4, 0.0625, 1e-3, 16)
    u = ri.random_spectrum(n, o.kept_modes(nc), 8.0, 11) * n
    fine = o.nbar(u, p)
    coarse = o.nbar(o.restrict_state(u, nc), pc)
    np.testing.assert_allclose(coarse, o.restrict_state(fine, nc), atol=1e-13 * np.max(np.abs(fine)))
    np.testing.assert_allclose(o.coarse_step_on_grid(u, p, n), o.coarse_step(u, p), atol=0)
    g = o.coarse_step_on_grid(u, p, nc)
    assert np.all(g[:, o.kept_modes(nc) + 1:] == 0)


def test_parareal_with_coarse_grid_terminates_finitely():
    n, nc, S = 32, 16, 4
    p = o.Params(n, 0.05, 1e-4, 0.1, 0.01, 8)
    u0 = ri.random_spectrum(n, 8, 16.0, 5) * 6.0
    ser = o.serial_fine(u0, p, S)
    res = o.parareal(u0, p, S, k_max=S, G=lambda x: o.coarse_step_on_grid(x, p, nc))
    scale = np.max(np.abs(ser))
    for k, U in enumerate(res.iterates):
        for m in range(min(k, S) + 1):
            assert np.max(np.abs(U[m] - ser[m])) < 1e-13 * scale, (k, m)
