"""Pins of the oracle's single curvilinear grid (no GPU).

The paper discretises on curvilinear grids by the mapping method (Section
"Discrete approximations": a smooth map x = G(r) from the unit square, the
equations transformed by the chain rule, conservative centred differences).
The oracle's operator J L u = sum_mn D_m (J g^mn D_n u) is pinned by:
  * a rotated box: the metric is the identity up to the side lengths, so L
    must equal the Cartesian 5-point operator (itself pinned by the sine
    closed forms) -- a wrong metric term or sign breaks this;
  * a smooth map of the unit square onto itself: the continuous eigenvalues
    are pi^2 (k^2 + l^2), and the second-order discrete ones must approach
    them at O(h^2);
  * the invariants: J L symmetric in plain sums (L symmetric in the
    J-weighted ones), L 1 = 0 away from the boundary;
  * the wave-solve against its modal closed form (the dense eigenvectors),
    and the J-weighted Rayleigh quotient of an eigenvector.
"""
import math

import numpy as np
import pytest

import ew_inputs
from oracle import oracle as O


def _dense(m):
    return np.stack([O.mapped_apply_L(m, e) for e in np.eye(m.size)], axis=1)


@pytest.mark.parametrize("theta", [0.0, 0.3, 2.0])
def test_rotated_box_is_the_cartesian_operator(theta):
    n1, n2, lx, ly = 11, 8, 1.0, 0.7
    m = O.MappedGrid((n1, n2), ew_inputs.mapped_vertices(n1, n2, "rotated_box", theta=theta, lx=lx, ly=ly))
    g = O.Grid((n1, n2), (lx, ly), 2)
    u = np.random.default_rng(0).standard_normal(m.size)
    a, b = O.mapped_apply_L(m, u), O.apply_L(g, u)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    prm = O.filter_params(9.0, 2, 30)
    a, b = O.mapped_filter_explicit(m, prm, u), O.filter_explicit(g, prm, u)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    np.testing.assert_allclose(O.mapped_jacobian(m), lx * ly, rtol=1e-13)


def test_conservative_form_is_symmetric_in_the_jacobian_weights():
    m = O.MappedGrid((12, 10), ew_inputs.mapped_vertices(12, 10, "square_warp", eps=0.12))
    L = _dense(m)
    JL = O.mapped_jacobian(m)[:, None] * L
    assert np.max(np.abs(JL - JL.T)) <= 1e-13 * np.max(np.abs(JL))
    assert np.max(np.abs(L - L.T)) > 1e-3 * np.max(np.abs(L))  # not symmetric without the weights


def test_constants_are_in_the_kernel_away_from_the_boundary():
    n = 14
    m = O.MappedGrid((n, n), ew_inputs.mapped_vertices(n, n, "square_warp", eps=0.1))
    Lu = O.mapped_apply_L(m, np.ones(m.size)).reshape(n, n)
    scale = np.max(np.abs(O.mapped_apply_L(m, np.arange(m.size, dtype=float))))
    assert np.max(np.abs(Lu[1:-1, 1:-1])) <= 1e-12 * scale


def test_second_order_convergence_to_the_square_spectrum():
    """A map of the unit square onto itself leaves the continuous spectrum
    pi^2 (k^2 + l^2); halving h must cut the error of the lowest eigenvalues by
    about 4 (measured 3.9 - 4.0 on the largest of them)."""
    exact = np.pi ** 2 * np.array([2.0, 5.0, 5.0, 8.0, 10.0, 10.0])
    err = []
    for n in (15, 31):
        m = O.MappedGrid((n, n), ew_inputs.mapped_vertices(n, n, "square_warp", eps=0.1))
        ev = np.sort(-np.linalg.eigvals(_dense(m)).real)[:6]
        err.append(np.max(np.abs(ev - exact) / exact))
    assert err[1] < 1e-2 and err[0] / err[1] > 3.5, err


def test_wave_solve_equals_the_modal_closed_form():
    m = O.MappedGrid((10, 8), ew_inputs.mapped_vertices(10, 8, "square_warp", eps=0.15))
    L = _dense(m)
    lam2, V = np.linalg.eig(-L)
    lam2, V = lam2.real, V.real
    prm = O.filter_params(7.0, 2, 40)
    beta = O.beta_tilde(np.sqrt(lam2), prm)
    v = np.random.default_rng(4).standard_normal(m.size)
    ref = V @ (beta * np.linalg.solve(V, v))
    got = O.mapped_filter_explicit(m, prm, v)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(v))


def test_weighted_rayleigh_quotient_of_an_eigenvector():
    m = O.MappedGrid((9, 11), ew_inputs.mapped_vertices(9, 11, "square_warp", eps=0.1))
    lam2, V = np.linalg.eig(-_dense(m))
    k = int(np.argsort(lam2.real)[3])
    assert abs(O.mapped_rayleigh_lambda(m, V[:, k].real) ** 2 - lam2[k].real) <= 1e-11 * lam2[k].real
