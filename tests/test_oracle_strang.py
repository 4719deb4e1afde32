"""Pins of the oracle's Strang-splitting solver (Algorithm 3) and of standard
parareal with a Strang coarse step (Sec. 6.2), against what the mathematics
fixes: the exact linear flow, the textbook midpoint rule it reduces to, its
second order, the invariants of the model and parareal's finite termination."""
import math

import numpy as np
from scipy.linalg import expm

import rsw_inputs as ri
from oracle import rsw as o
from test_oracle_coarse import _geostrophic_state


def _state(n, seed=1, amp=1.0):
    return amp * ri.random_spectrum(n, min(8, o.kept_modes(n)), 16.0, seed)


def test_strang_linear_part_is_exact():
    # N switched off: the two half steps compose to exp(dT (-L_k/eps + D_k)) per k,
    # here via scipy's matrix exponential of the 3x3 symbol.
    p = o.Params(32, 0.01, 1e-3, 0.0625, 1e-3, 8)
    u0 = _state(32)
    zero = lambda u, n: np.zeros_like(u)
    got = o.strang_propagate(u0, p, nl=zero)
    for k in range(p.H):
        A = -o.L_symbol(float(k)) / p.eps - p.nu * k ** 4 * np.eye(3)
        np.testing.assert_allclose(got[:, k], expm(p.dT * A) @ o.project(u0, 32)[:, k],
                                   atol=1e-13 * np.max(np.abs(u0)))


def test_strang_reduces_to_explicit_midpoint_rule():
    # eps = inf and nu = 0: the linear half steps are the identity and one step is
    # the textbook explicit midpoint rule u + h N(u + h/2 N(u)).
    p = o.Params(32, math.inf, 0.0, 0.01, 0.01, 8)
    x = o.project(_state(32, amp=20.0), 32)
    h = 0.01
    N = lambda y: o.nonlinear(y, 32)
    ref = x + h * N(x + h / 2 * N(x))
    np.testing.assert_allclose(o.strang_step(x, p, h), ref, atol=1e-15 * np.max(np.abs(ref)))


def test_strang_second_order_convergence():
    # Halving h: error ratio ~ 4 against the (separately pinned, fourth-order)
    # ETDRK4 propagator at a much smaller step.
    n = 32
    p = o.Params(n, 0.05, 1e-3, 0.05, 0.01, 8)
    u0 = _state(n, amp=30.0)
    ref = o.fine_propagate(u0, p, steps=256)
    errs = [o.parseval_norm(o.strang_propagate(u0, p, steps=s) - ref) for s in (8, 16, 32, 64)]
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(slopes) > 1.8 and max(slopes) < 2.3, (errs, slopes)


def test_strang_mean_height_and_geostrophic_state():
    # h_0 is invariant (every h-tendency is an x-derivative); a slow-mode-only
    # state has N = 0 and only decays as e^{-nu k^4 t}.
    p = o.Params(32, 0.01, 1e-4, 0.0625, 1e-3, 8)
    u0 = _state(32, amp=20.0)
    f = o.strang_propagate(u0, p)
    assert abs(f[2, 0] - u0[2, 0]) < 1e-14 * np.max(np.abs(u0))
    g0 = _geostrophic_state(32, 4)
    decay = np.exp(-p.nu * np.arange(p.H) ** 4 * p.dT)
    np.testing.assert_allclose(o.strang_propagate(g0, p), decay * g0, atol=1e-13)
    np.testing.assert_allclose(o.coarse_step_strang(g0, p), decay * g0, atol=1e-13)


def test_standard_parareal_finite_termination():
    # Eq. 3.1 with the Strang coarse step: U_n^k = F^n(u0) for n <= k.
    p = o.Params(32, 0.05, 1e-4, 0.1, 0.01, 8)
    u0 = _state(32, amp=8.0)
    S = 5
    G = lambda x: o.coarse_step_strang(x, p)
    ser = o.serial_fine(u0, p, S)
    res = o.parareal(u0, p, S, k_max=S, G=G)
    scale = np.max(np.abs(ser))
    for k, U in enumerate(res.iterates):
        for n in range(0, min(k, S) + 1):
            assert np.max(np.abs(U[n] - ser[n])) < 1e-13 * scale, (k, n)


def test_standard_parareal_error_falls_with_iterations():
    # A coarse step of a few eps on smooth data: the error against the serial fine
    # solution falls from one iteration to the next (Sec. 6.2's comparison runs).
    p = o.Params(32, 0.1, 1e-4, 0.2, 0.004, 8)
    u0 = _state(32, amp=4.0)
    S = 8
    ser = o.serial_fine(u0, p, S)
    res = o.parareal(u0, p, S, k_max=4, G=lambda x: o.coarse_step_strang(x, p))
    err = [float(np.max(o.physical_linf(U - ser, 32) / o.physical_linf(ser, 32))) for U in res.iterates]
    assert all(err[i + 1] < err[i] for i in range(len(err) - 1)), err


# ----------------------------------------------------------- integrating-factor RK4

def test_ifrk4_linear_part_is_exact():
    p = o.Params(32, 0.01, 1e-3, 0.0625, 1e-3, 8)
    u0 = _state(32)
    zero = lambda u, n: np.zeros_like(u)
    got = o.ifrk4_propagate(u0, p, nl=zero)
    for k in range(p.H):
        A = -o.L_symbol(float(k)) / p.eps - p.nu * k ** 4 * np.eye(3)
        np.testing.assert_allclose(got[:, k], expm(p.dT * A) @ o.project(u0, 32)[:, k],
                                   atol=1e-13 * np.max(np.abs(u0)))


def test_ifrk4_reduces_to_classical_rk4():
    # eps = inf and nu = 0: the integrating factor is the identity.
    p = o.Params(32, math.inf, 0.0, 0.01, 0.01, 8)
    x = o.project(_state(32, amp=20.0), 32)
    h = 0.01
    N = lambda y: o.nonlinear(y, 32)
    k1 = N(x)
    k2 = N(x + h / 2 * k1)
    k3 = N(x + h / 2 * k2)
    k4 = N(x + h * k3)
    ref = x + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    np.testing.assert_allclose(o.ifrk4_step(x, p, h), ref, atol=1e-15 * np.max(np.abs(ref)))


def test_ifrk4_fourth_order_and_invariants():
    n = 32
    p = o.Params(n, 0.05, 1e-3, 0.05, 0.01, 8)
    u0 = _state(n, amp=30.0)
    ref = o.fine_propagate(u0, p, steps=512)
    errs = [o.parseval_norm(o.ifrk4_propagate(u0, p, steps=s) - ref) for s in (8, 16, 32, 64)]
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(slopes) > 3.5, (errs, slopes)
    q = o.Params(32, 0.01, 1e-4, 0.0625, 1e-3, 8)
    f = o.ifrk4_propagate(u0, q)
    assert abs(f[2, 0] - u0[2, 0]) < 1e-14 * np.max(np.abs(u0))
    g0 = _geostrophic_state(32, 4)
    decay = np.exp(-q.nu * np.arange(q.H) ** 4 * q.dT)
    np.testing.assert_allclose(o.ifrk4_propagate(g0, q), decay * g0, atol=1e-13)
