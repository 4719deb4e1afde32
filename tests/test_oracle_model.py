"""Oracle pins for the spectral model (Sec. 6.1): eigen-structure, transforms,
the pseudo-spectral nonlinearity against a brute-force convolution, norms."""
import math

import numpy as np
import pytest

import rsw_inputs as ri
from oracle import rsw as o


@pytest.mark.parametrize("F", [1.0, 2.5])
def test_eigen_structure_matches_paper_formula(F):
    # Sec. 6.1: L(e^{ikx} r) = i omega e^{ikx} r with omega = alpha sqrt(1 + k^2/F),
    # alpha in {-1, 0, 1}; eigenvectors orthonormal (L_k skew-Hermitian).
    for k in [0, 1, 2, 7, 33, 500, -3]:
        om, V = o.L_eigen(float(k), F)
        sig = math.sqrt(1 + k * k / F)
        np.testing.assert_allclose(om, [-sig, 0.0, sig], rtol=0, atol=1e-13 * sig)
        L = o.L_symbol(float(k), F)
        np.testing.assert_allclose(L @ V, V @ np.diag(1j * om), atol=1e-13 * sig)
        np.testing.assert_allclose(V.conj().T @ V, np.eye(3), atol=1e-14)
        # skew-Hermitian symbol
        np.testing.assert_allclose(L.conj().T, -L, atol=0)


def test_eigen_slow_mode_closed_form():
    # The omega = 0 eigenvector is (0, ik, 1)/sqrt(1+k^2) up to a phase: v1 = 0 in it.
    for k in [0, 3, 40]:
        om, V = o.L_eigen(float(k))
        r0 = np.array([0, 1j * k, 1]) / math.sqrt(1 + k * k)
        assert abs(abs(np.vdot(r0, V[:, 1])) - 1.0) < 1e-14


def test_transform_convention_against_direct_sum():
    # u(x_j) = sum_{k=-N/2+1}^{N/2} u_k e^{i k x_j}, written as an O(N^2) sum.
    n = 16
    rng = np.random.default_rng(3)
    uh = (rng.standard_normal(n // 2 + 1) + 1j * rng.standard_normal(n // 2 + 1))
    uh[0] = uh[0].real
    uh[-1] = 0
    x = 2 * np.pi * np.arange(n) / n
    direct = np.zeros(n, dtype=complex)
    for k in range(-n // 2 + 1, n // 2 + 1):
        c = uh[k] if k >= 0 else np.conj(uh[-k])
        direct += c * np.exp(1j * k * x)
    np.testing.assert_allclose(o.synthesize(uh, n), direct.real, atol=1e-13)
    assert np.max(np.abs(direct.imag)) < 1e-13
    np.testing.assert_allclose(o.analyze(direct.real, n), uh, atol=1e-14)


def _truncated_convolution(u, n):
    """-sum_{k1+k2=k} [u1_{k1} i k2 u1_{k2}, u1_{k1} i k2 u2_{k2}, i k h_{k1} u1_{k2}],
    all |k1|, |k2|, |k| <= K: the exact dealiased nonlinearity, no transform."""
    K = o.kept_modes(n)

    def full(c, k):
        return c[k] if k >= 0 else np.conj(c[-k])

    out = np.zeros((3, n // 2 + 1), dtype=complex)
    for k in range(0, K + 1):
        s = np.zeros(3, dtype=complex)
        for k1 in range(-K, K + 1):
            k2 = k - k1
            if abs(k2) > K:
                continue
            v1a, v1b = full(u[0], k1), full(u[0], k2)
            v2b = full(u[1], k2)
            ha = full(u[2], k1)
            s[0] += v1a * 1j * k2 * v1b
            s[1] += v1a * 1j * k2 * v2b
            s[2] += 1j * k * ha * v1b
        out[:, k] = -s
    return out


@pytest.mark.parametrize("n", [8, 16, 32])
def test_pseudospectral_nonlinearity_equals_truncated_convolution(n):
    rng = np.random.default_rng(n)
    K = o.kept_modes(n)
    u = np.zeros((3, n // 2 + 1), dtype=complex)
    u[:, :K + 1] = rng.standard_normal((3, K + 1)) + 1j * rng.standard_normal((3, K + 1))
    u[:, 0] = u[:, 0].real
    got = o.nonlinear(u, n)
    ref = _truncated_convolution(u, n)
    np.testing.assert_allclose(got, ref, atol=1e-13 * np.max(np.abs(ref)))


def test_nonlinearity_analytic_case():
    # v1 = cos x, v2 = sin 2x, h = cos x: N = -(cos x (-sin x), cos x 2cos 2x, (cos^2 x)_x)
    #   = (sin 2x / 2, -(cos x + cos 3x), sin 2x)  -> coefficients at k = 1, 2, 3.
    n = 16
    u = np.zeros((3, 9), dtype=complex)
    u[0, 1] = 0.5
    u[1, 2] = -0.5j
    u[2, 1] = 0.5
    got = o.nonlinear(u, n)
    ref = np.zeros_like(got)
    ref[0, 2] = -0.25j   # sin 2x / 2 = (e^{2ix} - e^{-2ix})/(4i)
    ref[1, 1] = -0.5
    ref[1, 3] = -0.5
    ref[2, 2] = -0.5j    # sin 2x
    np.testing.assert_allclose(got, ref, atol=1e-15)


def test_projection_and_parseval():
    n = 32
    u = ri.random_spectrum(n, 15, 1e9, 5)
    u[:, 0] += 0.3j
    pu = o.project(u, n)
    assert np.all(pu[:, o.kept_modes(n) + 1:] == 0) and np.all(pu[:, 0].imag == 0)
    # Parseval: mean over the grid of sum_f u_f(x)^2 equals the squared norm.
    x = o.synthesize(pu, n)
    np.testing.assert_allclose(np.mean(np.sum(x ** 2, axis=0)), o.parseval_norm(pu) ** 2, rtol=1e-13)


def test_physical_linf_closed_form_and_axes():
    # The error metric of Sec. 6.2's experiments: the largest |u_f(x_j)| over the
    # grid points and the three fields, per state.  A two-mode state has it in
    # closed form: v1 = a cos x (u_1 = a/2) peaks at x = 0, h = b sin 2x
    # (u_2 = -i b/2) peaks at x = pi/4, both grid points for N = 8; v2 = 0.
    n = 8
    H = n // 2 + 1
    states = []
    for a, b in ((0.3, -1.7), (-2.5, 0.4), (0.0, 0.0)):
        u = np.zeros((3, H), dtype=np.complex128)
        u[0, 1] = a / 2.0
        u[2, 2] = -0.5j * b
        states.append(u)
    batch = np.stack(states)                       # (3 states, 3 fields, H)
    got = o.physical_linf(batch, n)
    assert got.shape == (3,)
    np.testing.assert_allclose(got, [1.7, 2.5, 0.0], rtol=1e-14, atol=1e-15)
    # a hand-written synthesis, term by term over -N/2 < k <= N/2, on a random
    # band-limited batch with two leading axes
    rng = np.random.default_rng(9)
    n = 16
    H = n // 2 + 1
    uh = rng.standard_normal((2, 2, 3, H)) + 1j * rng.standard_normal((2, 2, 3, H))
    uh[..., 0] = uh[..., 0].real
    uh[..., H - 1] = 0.0
    want = np.zeros((2, 2))
    for idx in np.ndindex(2, 2):
        best = 0.0
        for f in range(3):
            for j in range(n):
                x = 2.0 * math.pi * j / n
                s = uh[idx][f, 0].real
                for k in range(1, H - 1):
                    s += 2.0 * (uh[idx][f, k] * complex(math.cos(k * x), math.sin(k * x))).real
                best = max(best, abs(s))
        want[idx] = best
    np.testing.assert_allclose(o.physical_linf(uh, n), want, rtol=1e-13)
