"""Oracle pins for the fine propagator (ETDRK4, Cox & Matthews; named in Sec. 6.2):
phi-functions, the linear part solved exactly, reduction to classical RK4,
fourth order, and conservation of the mean height."""
import math

import mpmath
import numpy as np
import pytest
from scipy.linalg import expm

import rsw_inputs as ri
from oracle import rsw as o


def _mp_phi(z, j):
    """phi_j(z) = (e^z - sum_{n<j} z^n/n!) / z^j at 90 digits (the closed form
    cancels about 3*log10(1/|z|) digits near z = 0)."""
    mpmath.mp.dps = 90
    z = mpmath.mpc(z.real, z.imag)
    if z == 0:
        return complex(1 / mpmath.factorial(j))
    s = mpmath.exp(z)
    for n in range(j):
        s -= z ** n / mpmath.factorial(n)
    return complex(s / z ** j)


def test_phi_functions_against_high_precision():
    zs = np.array([0, 1e-9, 1e-3 + 2e-3j, -0.5, 0.99j, -0.999 + 0.01j, 1.0001, -2 + 17j,
                   -13.5 - 34j, -60 + 3j, 5 - 1j, -8.4 + 170j])
    got = o.phi123(zs)
    for j in range(3):
        ref = np.array([_mp_phi(z, j + 1) for z in zs])
        np.testing.assert_allclose(got[j], ref, rtol=3e-14, atol=0)


def _params(n=32, eps=0.05, nu=1e-3, dT=0.05, dt=0.01, m=16):
    return o.Params(n, eps, nu, dT, dt, m)


def _state(n, seed=1, amp=1.0):
    return amp * ri.random_spectrum(n, min(8, o.kept_modes(n)), 16.0, seed)


def test_linear_part_is_exact():
    # N switched off: F(u0) = exp(dT (-L_k/eps + D_k)) u0 per k, here via scipy's
    # matrix exponential of the 3x3 symbol (no eigendecomposition involved).
    p = _params(eps=0.01, dT=0.0625, dt=1e-3)
    u0 = _state(p.n_grid)
    zero = lambda u, n: np.zeros_like(u)
    got = o.fine_propagate(u0, p, nl=zero)
    ref = np.zeros_like(u0)
    for k in range(p.H):
        A = -o.L_symbol(float(k)) / p.eps - p.nu * k ** 4 * np.eye(3)
        ref[:, k] = expm(p.dT * A) @ o.project(u0, p.n_grid)[:, k]
    np.testing.assert_allclose(got, ref, atol=1e-13 * np.max(np.abs(u0)))
    # with nu = 0 the norm is conserved (L_k skew-Hermitian)
    p0 = _params(eps=0.01, nu=0.0, dT=0.0625, dt=1e-3)
    g0 = o.fine_propagate(u0, p0, nl=zero)
    assert abs(o.parseval_norm(g0) / o.parseval_norm(o.project(u0, 32)) - 1) < 1e-13


def test_reduces_to_classical_rk4_when_linear_part_vanishes():
    # eps = inf and nu = 0: the exponential weights become h/6, h/3, h/3, h/6.
    p = o.Params(32, math.inf, 0.0, 0.01, 0.01, 8)
    u = _state(32, amp=20.0)
    h = 0.01
    got = o.fine_step(o.project(u, 32), p, h)
    N = lambda x: o.nonlinear(x, 32)
    x = o.project(u, 32)
    k1 = N(x)
    k2 = N(x + h / 2 * k1)
    k3 = N(x + h / 2 * k2)
    k4 = N(x + h * k3)
    ref = x + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    np.testing.assert_allclose(got, ref, atol=1e-15 * np.max(np.abs(ref)))
    c = o.etdrk4_coefficients(p, h)
    np.testing.assert_allclose(c["f1"][3], h / 6 * np.eye(3), atol=1e-18)
    np.testing.assert_allclose(2 * c["f2"][3], h / 3 * np.eye(3), atol=1e-18)
    np.testing.assert_allclose(c["f3"][3], h / 6 * np.eye(3), atol=1e-18)
    np.testing.assert_allclose(c["Q"][3], h / 2 * np.eye(3), atol=1e-18)


def test_fourth_order_convergence():
    # Halving h in the regime h <= eps/4 on smooth data: error ratio ~ 16.
    n = 32
    p = o.Params(n, 0.05, 1e-3, 0.05, 0.01, 8)
    u0 = _state(n, amp=30.0)
    ref = o.fine_propagate(u0, p, steps=512)
    errs = []
    for steps in (4, 8, 16, 32):
        errs.append(o.parseval_norm(o.fine_propagate(u0, p, steps=steps) - ref))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(slopes) > 3.5, (errs, slopes)


@pytest.mark.parametrize("nu", [0.0, 1e-4])
def test_mean_height_is_invariant(nu):
    # Every h-tendency is an x-derivative and L_0 leaves h alone, so h_0 is constant.
    p = _params(nu=nu, eps=0.01, dT=0.0625, dt=1e-3)
    u0 = _state(p.n_grid, amp=20.0)
    f = o.fine_propagate(u0, p)
    assert abs(f[2, 0] - u0[2, 0]) < 1e-14 * np.max(np.abs(u0))
    assert abs(f[2, 0].imag) < 1e-15


def test_steps_rule():
    assert o.fine_steps(0.0625, 1e-3)[0] == 63
    assert o.fine_steps(10 / 256, 1e-4)[0] == 391
    assert o.fine_steps(10 / 512, 1e-5)[0] == 1954
    assert o.fine_steps(0.5, 0.1)[0] == 5   # exact division is not rounded up
