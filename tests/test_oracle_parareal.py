"""Oracle pins for parareal (Eq. 3.1, Algorithm 4): finite termination, exact
convergence when G = F, invariants, convergence on the small workload, and the
complexity model of Eq. 5.1 against the paper's printed example."""
import math
import os

import numpy as np
import pytest

import rsw_inputs as ri
from oracle import rsw as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small(n=16, slices=4):
    p = o.Params(n, 0.02, 1e-3, 0.05, 0.0125, 8)
    u0 = 2.0 * ri.random_spectrum(n, 5, 16.0, 21)
    return p, u0, slices


def test_finite_termination():
    # U_n^k = F^n(u0) for n <= k, so after S iterations parareal equals the serial
    # fine solution (follows from Eq. 3.1 by induction on n).
    p, u0, S = _small(slices=5)
    ser = o.serial_fine(u0, p, S)
    res = o.parareal(u0, p, S, k_max=S)
    scale = np.max(np.abs(ser))
    for k, U in enumerate(res.iterates):
        for n in range(0, min(k, S) + 1):
            assert np.max(np.abs(U[n] - ser[n])) < 1e-13 * scale, (k, n)
    assert np.max(np.abs(res.iterates[-1] - ser)) < 1e-13 * scale


def test_coarse_equal_to_fine_converges_in_one_iteration():
    p, u0, S = _small(slices=4)
    F = lambda x: o.fine_propagate(x, p)
    res = o.parareal(u0, p, S, k_max=2, F=F, G=F)
    ser = o.serial_fine(u0, p, S)
    np.testing.assert_allclose(res.iterates[0], ser, atol=1e-15)
    np.testing.assert_allclose(res.iterates[1], ser, atol=1e-14 * np.max(np.abs(ser)))
    assert res.changes[0] < 1e-14


def test_mean_height_through_parareal():
    p, u0, S = _small(slices=3)
    res = o.parareal(u0, p, S, k_max=2)
    for U in res.iterates:
        assert np.max(np.abs(U[:, 2, 0] - u0[2, 0].real)) < 1e-14 * np.max(np.abs(u0))


def test_stopping_rule_and_norm():
    a = np.zeros((2, 3, 5), dtype=complex)
    b = a.copy()
    a[0, 0, 1] = 1.0
    b[0, 0, 1] = 1.1
    a[1, 2, 0] = 2.0
    b[1, 2, 0] = 2.0
    # slice 0: |0.1| * sqrt(2) / (1.1 sqrt(2)); slice 1 unchanged
    assert math.isclose(o.rel_change_norm(b, a), 0.1 / 1.1, rel_tol=1e-14)
    z = np.zeros((1, 3, 5), dtype=complex)
    assert o.rel_change_norm(z, z) == 0.0
    p, u0, S = _small(slices=3)
    res = o.parareal(u0, p, S, k_max=5, tol=1e30)
    assert len(res.iterates) == 2   # stops after the first refinement


@pytest.mark.slow
def test_small_workload_converges():
    # N = 64, eps = 0.01, 16 slices, dt = 1e-3, M = 32: error to the serial fine
    # solution falls by more than an order of magnitude per iteration.
    w = ri.SMALL_N64
    p = o.Params(w.n_grid, w.eps, w.nu, w.dT, w.dt, w.m_quad)
    u0 = w.initial_state()
    res = o.parareal(u0, p, w.slices, w.k_max)
    ser = o.serial_fine(u0, p, w.slices)
    errs = [max(o.parseval_norm(U[n] - ser[n]) / o.parseval_norm(ser[n]) for n in range(1, w.slices + 1))
            for U in res.iterates]
    assert errs[0] < 0.05
    assert all(errs[i + 1] < 0.1 * errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-10


def test_complexity_model_matches_printed_example():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "eq51_speedup.txt")) if l.strip() and l[0] != "#"]
    for n_sl, m, it, printed, tol in rows:
        val = o.estimated_speedup(float(n_sl), float(m), float(it))
        assert abs(val - float(printed)) <= float(tol), val
    # Eq. 5.1's bound: speedup <= min(tau_f M / (tau_c (nu+1)), N / nu)
    for tf, tc in ((1.0, 1.0), (3.0, 1.0), (1.0, 0.2)):
        v = o.estimated_speedup(100, 400, 3, tf, tc)
        assert v <= min(tf * 400 / (tc * 4), 100 / 3) + 1e-12
