"""Pins of the oracle's wave-solve (one application of S) against the closed
forms of the paper's discrete analysis (no GPU)."""
import math

import numpy as np
import pytest

import ew_inputs
from oracle import oracle as O

CASES = [
    ((15, 11), (1.0, 1.3)),
    ((7, 9, 5), (1.0, 1.3, 0.8)),
]


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("n,length", CASES)
@pytest.mark.parametrize("scheme", ["explicit", "implicit"])
def test_single_mode_amplification(order, n, length, scheme):
    """S phi_k = beta~_d(lambda_k) phi_k (eqs. betad, correctedBeta, with the
    time correction eq. discreteExplicitLambdaTilde or eq. discreteCorr)."""
    g = O.Grid(n, length, order)
    if scheme == "explicit":
        prm = O.filter_params(9.0, 2, O.steps_per_period_cfl(g, 9.0, 0.8))
    else:
        prm = O.filter_params(9.0, 2, 10, adjust=True)
    for k in [(1,) * g.dim, (2, 3, 1)[:g.dim], tuple(g.n)]:
        phi = O.sine_mode(g, k)
        lam = math.sqrt(O.lambda2_closed_form(g, [k])[0])
        out = O.filter_apply(g, prm, phi, scheme)
        beta = O.beta_tilde(lam, prm, scheme)[0]
        assert np.max(np.abs(out - beta * phi)) < 1e-12


@pytest.mark.parametrize("order", [2, 4])
def test_dense_filter_operator(order):
    """S formed column by column on a tiny grid is symmetric, and its
    eigenvalues are beta~_d at every closed-form lambda (the discrete form of
    the theorem 'Eigenvalues of the EigenWave operator')."""
    g = O.Grid((5, 4), (1.0, 0.8), order)
    prm = O.filter_params(6.0, 1, O.steps_per_period_cfl(g, 6.0, 0.8))
    N = g.size
    S = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        S[:, j] = O.filter_explicit(g, prm, e)
    assert np.max(np.abs(S - S.T)) < 1e-14
    ev = np.sort(np.linalg.eigvalsh(0.5 * (S + S.T)))
    want = np.sort(O.beta_tilde(np.sqrt(O.spectrum(g)[0]), prm))
    np.testing.assert_allclose(ev, want, atol=1e-13)
    assert ev.min() >= -0.5 - 1e-2 and ev.max() <= 1.0 + 1e-12


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("scheme", ["explicit", "implicit"])
def test_random_input_matches_sine_basis(order, scheme):
    """On a random start vector, stepping the scheme equals applying the
    closed-form spectrum in the sine basis (DST)."""
    g = O.Grid((17, 12), (1.0, 1.5), order)
    v = ew_inputs.uniform_pm1(11, g.size)
    if scheme == "explicit":
        prm = O.filter_params(14.0, 1, O.steps_per_period_cfl(g, 14.0, 0.8))
    else:
        prm = O.filter_params(14.0, 1, 10, adjust=True)
    out = O.filter_apply(g, prm, v, scheme)
    ref = O.filter_closed_form(g, prm, v, 1, scheme)
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(v))


def test_symmetry_invariant_3d_order4():
    """(S u, w) = (u, S w) for the unweighted inner product."""
    g = O.Grid((9, 7, 6), (1.0, 0.9, 0.8), 4)
    prm = O.filter_params(10.0, 1, O.steps_per_period_cfl(g, 10.0, 0.8))
    u = ew_inputs.uniform_pm1(1, g.size)
    w = ew_inputs.uniform_pm1(2, g.size)
    a = np.dot(O.filter_explicit(g, prm, u), w)
    b = np.dot(u, O.filter_explicit(g, prm, w))
    assert abs(a - b) < 1e-13 * g.size


def test_cg_solve_matches_closed_form():
    """M^{-1} b by CG equals the sine-basis division by 1 + a lambda^2, and M's
    eigenvalues are 1 + a lambda^2 > 1 (eq. impMatrix, definite)."""
    g = O.Grid((11, 8, 7), (1.0, 1.0, 1.0), 4)
    a = 0.5 * 0.02 ** 2
    b = ew_inputs.uniform_pm1(5, g.size)
    x = O.cg_solve_M(g, a, b, tol=1e-15)
    np.testing.assert_allclose(x, O.implicit_solve_closed_form(g, a, b), atol=1e-13)
    assert np.dot(b, O.apply_M(g, a, b)) > np.dot(b, b)


def test_power_iteration_matches_closed_form_power():
    """Algorithm EigenWave (power iteration) for 40 iterations on the 2D unit
    square, order 2, omega = 20, FP64 explicit at CFL 0.8 (31x31 here, the
    63x63 case runs in the GPU tests): the iterate equals S^40 v / ||S^40 v||
    from the sine-basis closed form."""
    g = O.Grid((31, 31), (1.0, 1.0), 2)
    prm = O.filter_params(20.0, 1, O.steps_per_period_cfl(g, 20.0, 0.8))
    v0 = ew_inputs.uniform_pm1(ew_inputs.BASE_SEED, g.size)
    v, betas = O.power_iteration(lambda x: O.filter_explicit(g, prm, x), v0, 40)
    ref = O.filter_closed_form(g, prm, v0 / np.linalg.norm(v0), 40)
    ref /= np.linalg.norm(ref)
    assert np.max(np.abs(v - ref)) < 1e-11
    lam = O.rayleigh_lambda(g, v)
    lam2 = O.spectrum(g)[0]
    assert math.sqrt(lam2.min()) <= lam <= math.sqrt(lam2.max())
