"""Pins of the oracle's Krylov eigen-solver, multigrid and learned-smoother
pieces (no GPU)."""
import math

import numpy as np
import pytest

import ew_inputs
from oracle import oracle as O


def _nearest_levels(g, prm, n_wanted, scheme="explicit"):
    """The n_wanted closed-form lambda with the largest beta~_d."""
    lam = np.sqrt(O.spectrum(g)[0])
    b = O.beta_tilde(lam, prm, scheme)
    idx = np.argsort(-b)[:n_wanted]
    return np.sort(lam[idx]), np.sort(b[idx])[::-1]


@pytest.mark.parametrize("order,scheme", [(4, "explicit"), (2, "implicit")])
def test_krylov_schur_finds_closed_form_eigenpairs(order, scheme):
    g = O.Grid((31, 47), (1.0, 1.5), order)
    omega = 25.0
    if scheme == "explicit":
        prm = O.filter_params(omega, 2, O.steps_per_period_cfl(g, omega, 0.8))
    else:
        prm = O.filter_params(omega, 4, 10, adjust=True)
    v0 = ew_inputs.start_block(3, g.size, 2)
    theta, X, nmv = O.krylov_schur_eigs(lambda v: O.filter_apply(g, prm, v, scheme), v0, 6, 30,
                                        tol=1e-10, max_matvecs=400)
    assert len(theta) == 6
    want_lam, want_beta = _nearest_levels(g, prm, 6, scheme)
    np.testing.assert_allclose(theta, want_beta, atol=1e-9)
    lam = np.sort([O.rayleigh_lambda(g, X[:, j]) for j in range(6)])
    np.testing.assert_allclose(lam, want_lam, rtol=1e-10)
    for j in range(6):
        l = O.rayleigh_lambda(g, X[:, j])
        assert O.eig_res(g, l, X[:, j]) < 1e-7


def test_cgs2_orthogonalises_to_rounding_on_nearly_dependent_vectors():
    """Gram-Schmidt twice ("twice is enough", Kahan-Parlett): against an
    orthonormal basis the projected vector is orthogonal to rounding even when
    w lies almost in span(V), where one classical pass leaves an error of
    about eps ||w|| / ||w_perp||; and w = w_perp + V h exactly up to rounding."""
    rng = np.random.default_rng(3)
    N, m = 4000, 24
    V, _ = np.linalg.qr(rng.standard_normal((N, m)))
    for gap in (1e-2, 1e-6, 1e-9):
        w = V @ rng.standard_normal(m) + gap * rng.standard_normal(N)
        wp, h = O._cgs2(V, w)
        eps = np.finfo(float).eps
        assert np.max(np.abs(V.T @ wp)) <= 50 * eps * np.linalg.norm(wp)
        assert np.linalg.norm(w - wp - V @ h) <= 50 * eps * np.linalg.norm(w)
        # one pass is not enough once the gap is small (what the second pass is for)
        one = w - V @ (V.T @ w)
        if gap <= 1e-6:
            assert np.max(np.abs(V.T @ one)) > 50 * eps * np.linalg.norm(one)


def test_eigenspace_distance_of_multiple_eigenvalue():
    """evect-err by projection onto a multiple eigenspace: any combination of
    the (3,1) and (1,3) square modes is at distance 0, another mode is not."""
    g = O.Grid((15, 15), (1.0, 1.0), 2)
    a, b = O.sine_mode(g, (3, 1)), O.sine_mode(g, (1, 3))
    basis = np.column_stack([a, b])
    assert O.eigenspace_distance(0.3 * a - 2.0 * b, basis) < 1e-13
    assert O.eigenspace_distance(O.sine_mode(g, (2, 2)), basis) > 0.5


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 4), (3, 2)])
def test_multigrid_converges_to_exact_solve(dim, order):
    n = (31, 31, 31)[:dim]
    g = O.Grid(n, (1.0,) * dim, order)
    a = 0.5 * (2 * math.pi / (20.0 * 10)) ** 2
    b = ew_inputs.uniform_pm1(7, g.size)
    exact = O.implicit_solve_closed_form(g, a, b)
    x, hist = O.mg_solve(g, a, b, ncycles=12)
    rho = (hist[-1] / hist[0]) ** (1 / 12)
    assert rho < 0.25
    assert np.max(np.abs(x - exact)) < 1e-9 * np.max(np.abs(exact))


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 2), (2, 4), (3, 4)])
def test_red_black_multigrid_converges_to_exact_solve_and_beats_jacobi(dim, order):
    """Multi-colour Gauss-Seidel smoothing (red-black at second order, three
    colours at fourth order): the same exact solve (the sine-basis closed form
    of M^-1), and a smaller contraction per cycle than damped Jacobi on a
    strongly elliptic system (a / h^2 >> 1)."""
    n = (63, 63) if dim == 2 else (31, 31, 31)
    g = O.Grid(n, (1.0,) * dim, order)
    a = 0.5 * (2 * math.pi / (12.0 * 10)) ** 2   # the 2D scaling runs' implicit step
    b = ew_inputs.uniform_pm1(8, g.size)
    exact = O.implicit_solve_closed_form(g, a, b)
    xr, hr = O.mg_solve(g, a, b, ncycles=12, red_black=True)
    xj, hj = O.mg_solve(g, a, b, ncycles=12)
    assert np.max(np.abs(xr - exact)) < 1e-9 * np.max(np.abs(exact))
    assert (hr[-1] / hr[0]) < 0.25 * (hj[-1] / hj[0])


def _jacobi_as_net(g, a, wJ=0.8):
    """Learned weights that make the learned correction equal to damped Jacobi:
    W1 = identity tap on channel 0, W2 = (wJ / D) centre tap on channel 0."""
    d0 = 2.0 if g.order == 2 else 2.5
    D = 1 + a * sum(d0 / h ** 2 for h in g.h)
    w = np.zeros(O.NET_WEIGHTS)
    w[13] = 1.0
    w[8 * 27 + 13] = wJ / D
    return w


def test_learned_path_reduces_to_jacobi():
    g = O.Grid((15, 15, 15), (1.0, 1.0, 1.0), 4)
    a = 0.5 * (2 * math.pi / 800.0) ** 2
    b = ew_inputs.uniform_pm1(9, g.size)
    w = _jacobi_as_net(g, a)
    nets = np.stack([w, _jacobi_as_net(O.Grid((7, 7, 7), (1.0,) * 3, 4), a)])
    x1, h1 = O.mg_solve(g, a, b, ncycles=3)
    x2, h2 = O.mg_solve(g, a, b, ncycles=3, net=nets)
    assert np.max(np.abs(x1 - x2)) < 1e-13
    np.testing.assert_allclose(h1, h2, rtol=0, atol=1e-13 * h1[0])


def test_conv_net_forward_special_cases():
    """Single-tap kernels act as shifts with zero fill: W1 tap (dz,dy,dx) =
    (0,0,1) on channel 2, W2 tap (1,0,0) on channel 2 gives y(x) = r(x + ex + ez)."""
    n3 = (5, 4, 3)
    r = ew_inputs.uniform_pm1(4, 60).reshape(3, 4, 5)
    w = np.zeros(O.NET_WEIGHTS)
    tap = lambda dz, dy, dx: (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
    w[2 * 27 + tap(0, 0, 1)] = 1.0
    w[8 * 27 + 2 * 27 + tap(1, 0, 0)] = 2.0
    _, y = O.conv_net_forward(n3, w, r.reshape(-1))
    ref = np.zeros_like(r)
    ref[:-1, :, :-1] = 2.0 * r[1:, :, 1:]
    np.testing.assert_allclose(y.reshape(r.shape), ref, atol=1e-15)


def test_conv_net_gradient_matches_finite_differences():
    """Backward of the smoother loss against central finite differences of the
    oracle's own forward pass (FP64)."""
    g = O.Grid((6, 5, 4), (1.0, 0.9, 0.8), 4)
    a = 0.5 * 0.05 ** 2
    r = ew_inputs.uniform_pm1(12, g.size)
    w = ew_inputs.learned_init(13, 0.2)
    loss, gw = O.smoother_loss(g, a, w, r)
    eps = 1e-6
    for idx in [0, 13, 26, 100, 216, 229, 300, 431]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += eps
        wm[idx] -= eps
        fd = (O.smoother_loss(g, a, wp, r)[0] - O.smoother_loss(g, a, wm, r)[0]) / (2 * eps)
        assert abs(fd - gw[idx]) < 1e-6 * max(1.0, abs(fd))


def test_implicit_filter_with_multigrid_tends_to_exact():
    """The multigrid-based implicit wave-solve converges to the exactly solved
    one as the V-cycles per system grow."""
    g = O.Grid((15, 15, 15), (1.0, 1.0, 1.0), 4)
    prm = O.filter_params(12.0, 1, 10, adjust=True)
    v = ew_inputs.uniform_pm1(41, g.size)
    exact = O.filter_implicit(g, prm, v)
    e2 = np.max(np.abs(O.filter_implicit_mg(g, prm, v, ncycles=2) - exact))
    e12 = np.max(np.abs(O.filter_implicit_mg(g, prm, v, ncycles=12) - exact))
    assert e12 < 1e-9 and e12 < e2 / 1e5


def test_previous_solution_guess_starts_from_the_closed_form_residual():
    """With the previous system's solution as the initial guess (reading of the
    unstated guess), system n starts from the residual 2 (W^n - W^{n-1}) when
    the systems are solved (nearly) exactly, independent of h; the converged
    wave-solve is the exactly solved one either way."""
    g = O.Grid((15, 31), (1.0, 1.7), 4)
    prm = O.filter_params(12.0, 1, 10, adjust=True)
    v = ew_inputs.uniform_pm1(42, g.size)
    exact = O.filter_implicit(g, prm, v)
    a = 0.5 * prm["dt"] ** 2
    out, hists = O.filter_implicit_mg(g, prm, v, ncycles=25, guess="previous", return_hist=True)
    assert np.max(np.abs(out - exact)) < 1e-10 * np.max(np.abs(exact))
    # the time levels of the exactly solved scheme, from its own recurrence
    w = [v.copy(), O.cg_solve_M(g, a, v)]
    for n in range(1, 5):
        y = O.cg_solve_M(g, a, 2.0 * w[n])
        w.append(y - w[n - 1])
    for n in range(2, 5):     # the second system starts from 2 W^1 (y_0 under W^{-1} = W^1)
        want = np.linalg.norm(2.0 * (w[n] - w[n - 1]))
        assert hists[n][0] == pytest.approx(want, rel=1e-8)
    # and the rhs guess starts much higher on this grid (residual a L_h 2 W^n)
    _, hr = O.filter_implicit_mg(g, prm, v, ncycles=25, return_hist=True)
    assert hr[3][0] > 3.0 * hists[3][0]
