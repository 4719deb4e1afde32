"""Plants plausible mistakes in the oracle (CPU only) and checks that a pin fails
for each: the pins must be able to tell a wrong oracle from a right one."""
import numpy as np
import pytest

from oracle import rsw
import test_oracle_coarse as tc
import test_oracle_fine as tf
import test_oracle_model as tm
import test_oracle_parareal as tp
import test_oracle_strang as ts


def _bad_nl_sign(u, n):
    out = _orig["nonlinear"](u, n)
    out[..., 2, :] *= -1.0
    return out


def _bad_nl_no_derivative(u, n):
    k = np.arange(u.shape[-1])
    out = _orig["nonlinear"](u, n)
    with np.errstate(divide="ignore", invalid="ignore"):
        out[..., 2, 1:] = out[..., 2, 1:] / (1j * k[1:])
    return out


def _bad_phi(z):
    a, b, c = _orig["phi123"](z)
    return a, b, c * (1 + 1e-6)


def _bad_etd(p, h):
    c = dict(_orig["etdrk4_coefficients"](p, h))
    c["f2"] = c["f2"] * 1.5          # wrong weight on N(a) + N(b)
    return c


def _bad_expL(p, s):
    return _orig["expL"](p, -s)      # phases of e^{sL} and e^{-sL} swapped


def _bad_apply(m, u):
    return np.einsum("kji,...jk->...ik", m, u)   # transposed operand


def _bad_linf_grid_axis_only(u, n):
    return np.max(np.abs(rsw.synthesize(u, n)), axis=-1)       # reduces the grid axis only


def _bad_linf_unscaled(u, n):
    return np.max(np.abs(np.fft.irfft(u, n=n, axis=-1)), axis=(-2, -1))   # drops the factor N


def _bad_quadrature(p):
    s, w = _orig["quadrature"](p)
    return s + p.window / p.m_quad / 2, w        # nodes shifted by half a spacing


def _bad_strang_one_half_step(u, p, h, nl=None):
    nl = nl or rsw.nonlinear
    w = rsw._apply(rsw.linear_matrices(p, h / 2.0), u)   # second linear half step dropped
    k1 = nl(w, p.n_grid)
    return w + h * nl(w + h / 2 * k1, p.n_grid)


def _bad_strang_stage_from_u(u, p, h, nl=None):
    nl = nl or rsw.nonlinear
    E2 = rsw.linear_matrices(p, h / 2.0)
    w = rsw._apply(E2, u)
    k1 = nl(w, p.n_grid)
    k2 = nl(u + h / 2 * k1, p.n_grid)                    # midpoint stage built on u, not w
    return rsw._apply(E2, w + h * k2)


def _bad_ifrk4_stage(u, p, h, nl=None):
    nl = nl or rsw.nonlinear
    E2 = rsw.linear_matrices(p, h / 2.0)
    E = rsw.linear_matrices(p, h)
    k1 = nl(u, p.n_grid)
    k2 = nl(rsw._apply(E2, u + h / 2 * k1), p.n_grid)
    k3 = nl(u + h / 2 * k2, p.n_grid)                    # third stage without the half-step factor
    k4 = nl(rsw._apply(E, u) + h * rsw._apply(E2, k3), p.n_grid)
    return rsw._apply(E, u) + h / 6 * (rsw._apply(E, k1) + 2 * rsw._apply(E2, k2 + k3) + k4)


_orig = {name: getattr(rsw, name) for name in
         ("nonlinear", "phi123", "etdrk4_coefficients", "expL", "_apply", "quadrature", "strang_step", "ifrk4_step",
          "physical_linf")}

CASES = [
    ("nonlinear", _bad_nl_sign, tm.test_nonlinearity_analytic_case, ()),
    ("nonlinear", _bad_nl_no_derivative, tm.test_pseudospectral_nonlinearity_equals_truncated_convolution, (16,)),
    ("phi123", _bad_phi, tf.test_phi_functions_against_high_precision, ()),
    ("etdrk4_coefficients", _bad_etd, tf.test_reduces_to_classical_rk4_when_linear_part_vanishes, ()),
    ("expL", _bad_expL, tc.test_nbar_equals_brute_force_triad_sum, (8, 6, 3.0)),
    ("expL", _bad_expL, tc.test_coarse_step_linear_part_exact, ()),
    ("_apply", _bad_apply, tf.test_linear_part_is_exact, ()),
    ("quadrature", _bad_quadrature, tc.test_quadrature_weights_sum_to_one, (32,)),
    ("strang_step", _bad_strang_one_half_step, ts.test_strang_linear_part_is_exact, ()),
    ("strang_step", _bad_strang_stage_from_u, ts.test_strang_second_order_convergence, ()),
    ("ifrk4_step", _bad_ifrk4_stage, ts.test_ifrk4_fourth_order_and_invariants, ()),
    ("physical_linf", _bad_linf_grid_axis_only, tm.test_physical_linf_closed_form_and_axes, ()),
    ("physical_linf", _bad_linf_unscaled, tm.test_physical_linf_closed_form_and_axes, ()),
]


@pytest.mark.parametrize("name,bad,pin,args", CASES, ids=[f"{c[0]}-{c[1].__name__}" for c in CASES])
def test_pin_catches_planted_mistake(monkeypatch, name, bad, pin, args):
    pin(*args)                       # passes on the correct oracle
    monkeypatch.setattr(rsw, name, bad)
    with pytest.raises((AssertionError, FloatingPointError, ValueError)):
        pin(*args)


def test_finite_termination_catches_wrong_correction(monkeypatch):
    # Using the new coarse value in place of the old one in Eq. 3.1 breaks finite termination.
    orig = rsw.parareal

    def bad_parareal(u0, p, slices, k_max, tol=0.0, F=None, G=None):
        F = F or (lambda x: rsw.fine_propagate(x, p))
        G = G or (lambda x: rsw.coarse_step(x, p))
        U = [rsw.project(u0, p.n_grid)]
        for n in range(1, slices + 1):
            U.append(G(U[n - 1]))
        U = np.stack(U)
        res = rsw.PararealResult([U], [])
        for _ in range(k_max):
            f_old = F(U[:-1])
            new = [U[0]]
            for n in range(1, slices + 1):
                g_new = G(new[n - 1])
                new.append(g_new + f_old[n - 1] - g_new * 0.999)
            U = np.stack(new)
            res.iterates.append(U)
            res.changes.append(0.0)
        return res

    tp.test_finite_termination()
    monkeypatch.setattr(rsw, "parareal", bad_parareal)
    with pytest.raises(AssertionError):
        tp.test_finite_termination()
    monkeypatch.setattr(rsw, "parareal", orig)
