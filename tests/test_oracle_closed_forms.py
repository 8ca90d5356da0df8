"""Pins of the oracle's spatial operator and filter parameters against what the
paper prints and what the mathematics fixes (no GPU)."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                lam, mult = line.split()
                rows.append((float(lam), int(mult)))
    return rows


def _levels(g, lo, hi):
    """Distinct closed-form lambda_h in [lo, hi] with their multiplicities."""
    lam = np.sqrt(O.spectrum(g)[0])
    lam = np.sort(lam[(lam >= lo) & (lam <= hi)])
    levels = []
    for v in lam:
        if levels and abs(v - levels[-1][0]) < 1e-9 * v:
            levels[-1][1] += 1
        else:
            levels.append([v, 1])
    return levels


@pytest.mark.parametrize("fixture,n,length,lo,hi", [
    ("square128_order2_lambda.txt", (127, 127), (1.0, 1.0), 7.0, 20.2),
    ("box2_order2_lambda.txt", (19, 19, 19), (1.0, 1.0, 1.0), 5.4, 14.3),
])
def test_closed_form_matches_paper_tables(fixture, n, length, lo, hi):
    """The closed-form Dirichlet eigenvalues reproduce the paper's printed
    eigenvalue tables (6 decimals) with the printed multiplicities."""
    g = O.Grid(n, length, 2)
    want = _read_golden(fixture)
    got = _levels(g, lo, hi)
    assert len(got) == len(want)
    for (gl, gm), (wl, wm) in zip(got, want):
        assert abs(gl - wl) <= 5e-7 + 1e-9 * wl
        assert gm == wm


@pytest.mark.parametrize("fixture,n", [
    ("square128_order2_index.txt", (127, 127)),
    ("box2_order2_index.txt", (19, 19, 19)),
])
def test_closed_form_counts_the_eigenvalues_below_each_level(fixture, n):
    """The paper's index k of the closest true eigenvalue (same tables, the
    true eigenvalues sorted from k = 0) fixes how many eigenvalues of the whole
    discrete spectrum lie below each printed level: a closed form that dropped
    or doubled a mode family anywhere below the printed levels fails it."""
    g = O.Grid(n, (1.0,) * len(n), 2)
    lam = np.sort(np.sqrt(O.spectrum(g)[0]))
    with open(os.path.join(GOLDEN, fixture)) as f:
        rows = [line.split() for line in f if line.strip() and not line.startswith("#")]
    assert len(rows) == 27
    for j, lv, k, m in rows:
        lv, k, m = float(lv), int(k), int(m)
        below = int(np.sum(lam < lv - 5e-7))
        at = int(np.sum(np.abs(lam - lv) <= 5e-7 + 1e-9 * lv))
        assert at == m, (j, lv, at, m)
        assert below <= k <= below + m - 1, (j, lv, below, k)


def _dense(g, op):
    N = g.size
    A = np.empty((N, N))
    e = np.zeros(N)
    for j in range(N):
        e[:] = 0.0
        e[j] = 1.0
        A[:, j] = op(e)
    return A


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("n,length", [((6, 5), (1.0, 1.4)), ((4, 5, 3), (0.7, 1.0, 1.2))])
def test_dense_laplacian_spectrum(order, n, length):
    """-L_h formed column by column is symmetric positive definite and its
    eigenvalues (library eigensolver) are the closed-form lambda^2: this pins
    the stencil coefficients, the spacing and the odd-reflection closure."""
    g = O.Grid(n, length, order)
    A = -_dense(g, lambda e: O.apply_L(g, e))
    assert np.max(np.abs(A - A.T)) <= 1e-12 * np.max(np.abs(A))
    ev = np.sort(np.linalg.eigvalsh(A))
    cf = np.sort(O.spectrum(g)[0])
    assert ev[0] > 0
    np.testing.assert_allclose(ev, cf, rtol=1e-12, atol=1e-9)
    assert cf[-1] <= O.spectral_radius_bound(g)


@pytest.mark.parametrize("order", [2, 4])
def test_sine_mode_is_eigenvector(order):
    g = O.Grid((13, 9), (1.0, 0.6), order)
    for k in [(1, 1), (3, 7), (13, 9)]:
        phi = O.sine_mode(g, k)
        lam2 = O.lambda2_closed_form(g, [k])[0]
        np.testing.assert_allclose(O.apply_L(g, phi), -lam2 * phi, atol=1e-10 * lam2)


def test_order4_closure_is_fourth_order_accurate():
    """Interior and boundary rows of the order-4 operator converge at 4th order
    on a smooth function vanishing with its second derivative on the wall."""
    errs = []
    for n in (31, 63):
        g = O.Grid((n, n), (1.0, 1.0), 4)
        x = np.arange(1, n + 1) * g.h[0]
        X, Y = np.meshgrid(x, x, indexing="xy")
        u = np.sin(math.pi * X) * np.sin(2 * math.pi * Y) * (1 + 0.0 * X)
        exact = -(math.pi ** 2 + 4 * math.pi ** 2) * u
        errs.append(np.max(np.abs(O.apply_L(g, u.reshape(-1)) - exact.reshape(-1))))
    assert errs[0] / errs[1] > 14.0


@pytest.mark.parametrize("Nt", [5, 10, 36, 176])
def test_alpha_d_gives_unit_peak(Nt):
    """alpha_d (eq. alphad) makes the discrete filter reach one with zero slope
    at lambda~ = omega (the property the paper states for it)."""
    prm = O.filter_params(20.0, 1, Nt)
    w = prm["omega"]
    assert abs(O.beta_d(w, prm)[0] - 1.0) < 1e-13
    d = 1e-5 * w
    slope = (O.beta_d(w + d, prm)[0] - O.beta_d(w - d, prm)[0]) / (2 * d)
    assert abs(slope) * w < 1e-7


def test_alpha_d_half_breaks_peak():
    """With the continuous 1/4 (alpha = 1/2) the trapezoid sum still equals one
    at lambda = omega but its maximum moves off omega: alpha_d is what puts the
    maximum there."""
    prm = O.filter_params(20.0, 1, 10)
    prm_half = dict(prm)
    n = np.arange(prm["Nt"] + 1)
    sigma = np.full(prm["Nt"] + 1, prm["dt"])
    sigma[0] = sigma[-1] = prm["dt"] / 2
    prm_half["c"] = (2 / prm["Tf"]) * sigma * (np.cos(20.0 * n * prm["dt"]) - 0.25)
    d = 1e-5 * 20.0
    slope = (O.beta_d(20.0 + d, prm_half)[0] - O.beta_d(20.0 - d, prm_half)[0]) / (2 * d)
    assert abs(slope) * 20.0 > 1e-3


def test_quadrature_weights_sum():
    """Trapezoid weights: (2/T_f) sum sigma_n = 2 and sum c_n = beta_d(0)."""
    prm = O.filter_params(13.0, 3, 40)
    Nt, dt = prm["Nt"], prm["dt"]
    sigma = np.full(Nt + 1, dt)
    sigma[0] = sigma[-1] = dt / 2
    assert abs(2 / prm["Tf"] * sigma.sum() - 2.0) < 1e-13
    assert abs(prm["c"].sum() - O.beta_d(0.0, prm)[0]) < 1e-13


def test_continuous_filter_properties():
    """beta (eq. filterThreeSincs) lies in [-1/2, 1], peaks at 1 for lambda =
    omega, equals -1/2 at lambda = 0 for integer N_p, and matches the integral
    definition eq. filterFunction by brute-force quadrature."""
    omega = 7.0
    for Np in (1, 2, 5):
        Tf = Np * 2 * math.pi / omega
        lam = np.linspace(0, 6 * omega, 3001)
        b = O.beta_continuous(lam, omega, Tf)
        assert b.min() >= -0.5 - 1e-12 and b.max() <= 1 + 1e-12
        assert abs(O.beta_continuous(omega, omega, Tf) - 1.0) < 1e-12
        assert abs(O.beta_continuous(0.0, omega, Tf) + 0.5) < 1e-12
        t = np.linspace(0, Tf, 200001)
        for l in (0.3 * omega, 0.97 * omega, 2.2 * omega):
            f = (np.cos(omega * t) - 0.25) * np.cos(l * t)
            integral = (2 / Tf) * np.trapezoid(f, t)
            assert abs(integral - O.beta_continuous(l, omega, Tf)) < 1e-8


def test_simultaneous_iteration_worked_example():
    """The worked example of the simultaneous-iteration rate (Section
    "Estimating the EigenWave convergence rate based on simultaneous
    iteration", eq. subSpaceIterationEigenWaveCR, with omega = 1 and N_p = 1):
    a requested level beta_r of about 0.8 gives CR = beta(1 + 2 dw) /
    beta(1 + dw) of about 0.4, dw defined by beta(1 + dw) = beta_r.  The
    printed dw (about 0.375) is read as the width 2 dw of the interval
    [1 - dw, 1 + dw]: the definition gives dw = 0.182.  The paper also states
    that the rate is essentially independent of N_p while dw shrinks as
    1 / N_p (so N_r(N_p) is about N_r(1) / N_p)."""
    from scipy.optimize import brentq
    crs, widths = [], []
    for Np in (1, 2, 4, 8):
        Tf = Np * 2 * math.pi

        def beta(l):
            return float(O.beta_continuous(l, 1.0, Tf))
        dw = brentq(lambda d: beta(1.0 + d) - 0.8, 1e-9, 0.9 / Np)  # the first crossing past the peak
        crs.append(beta(1.0 + 2 * dw) / beta(1.0 + dw))
        widths.append(dw * Np)
    assert abs(crs[0] - 0.4) < 0.05
    assert abs(2 * widths[0] - 0.375) < 0.02
    assert max(crs) - min(crs) < 0.02
    assert max(widths) - min(widths) < 0.02 * widths[0]


def test_discrete_filter_tends_to_continuous():
    """beta_d -> beta as N_t grows (the discrete-analysis remark)."""
    omega = 9.0
    lam = np.linspace(0.1, 3 * omega, 50)
    errs = []
    for Nt in (40, 80, 160):
        prm = O.filter_params(omega, 1, Nt)
        errs.append(np.max(np.abs(O.beta_tilde(lam, prm) - O.beta_continuous(lam, omega, prm["Tf"]))))
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3


@pytest.mark.parametrize("n_its", [6, 10, 15])
def test_adjusted_omega(n_its):
    """omega~ (eq. adjustedOmega) solves eq. modifiedFrequencyEqn, and the
    time-corrected implicit filter with omega~ peaks (value 1, zero slope) at
    lambda = omega."""
    omega = 12.0
    wt = O.adjusted_omega(omega, n_its)
    dtt = 2 * math.pi / (wt * n_its)
    lhs = 2 / dtt * math.asin((omega * dtt / 2) / math.sqrt(1 + (omega * dtt) ** 2 / 2))
    assert abs(lhs - wt) < 1e-12 * omega
    prm = O.filter_params(omega, 1, n_its, adjust=True)
    assert abs(prm["omega"] - wt) < 1e-14 * omega
    assert abs(O.beta_tilde(omega, prm, "implicit")[0] - 1.0) < 1e-12
    d = 1e-5 * omega
    s = (O.beta_tilde(omega + d, prm, "implicit")[0] - O.beta_tilde(omega - d, prm, "implicit")[0])
    assert abs(s / (2 * d)) * omega < 1e-6


def test_lambda_tilde_limits():
    """Both time corrections tend to lambda as dt -> 0 with the textbook
    second-order error, and the explicit one is the leapfrog dispersion
    relation cos(lambda~ dt) = 1 - (lambda dt)^2 / 2."""
    lam = 5.0
    for dt in (1e-2, 1e-3):
        le = O.lambda_tilde_explicit(lam, dt)
        li = O.lambda_tilde_implicit(lam, dt)
        assert abs(le - lam) < lam ** 3 * dt ** 2
        assert abs(li - lam) < lam ** 3 * dt ** 2
        assert abs(math.cos(le * dt) - (1 - (lam * dt) ** 2 / 2)) < 1e-14
        # implicit: cos(li dt) = 1 / (1 + (lam dt)^2 / 2)
        assert abs(math.cos(li * dt) - 1 / (1 + (lam * dt) ** 2 / 2)) < 1e-14


def test_cfl_steps_match_configuration_notes():
    """Steps per period at CFL 0.8 for the unit-square 63x63 order-2 case: 36."""
    g = O.Grid((63, 63), (1.0, 1.0), 2)
    assert O.steps_per_period_cfl(g, 20.0, 0.8) == 36
