"""Pins of the oracle's Neumann faces (no GPU).

The paper treats a Neumann face as a symmetry plane (Section "Numerical
results", the double ellipsoid: Neumann conditions on the lower boundary,
which is a symmetry plane).  The oracle closes such a face by the even
reflection about its wall point (u_{-j} = u_{j}, the wall point active) and a
Dirichlet face by the odd reflection.  What pins it:

  * the symmetry plane itself: S of a vector that is symmetric about the
    centre of a Dirichlet box, restricted to one half, equals S on the half
    box whose face at the centre is a Neumann face -- the Dirichlet wave-solve
    is pinned independently (sine-basis closed forms, the paper's tables);
  * the spectrum of the dense L_h on tiny boxes (every column from the C
    stencil) against the textbook tensor sine / cosine spectrum of each face
    pair, and each mode against L_h pointwise;
  * the invariants: L_h symmetric in the trapezoid weights (not in the plain
    sums once a face is Neumann), L_h 1 = 0 on an all-Neumann box;
  * the weighted Rayleigh quotient of a mode is its eigenvalue.
A wrong mirror index, a sign, or a dropped ghost layer changes the spectrum
and breaks the symmetry-plane identity.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

BCS_2D = [("N", "D", "D", "D"), ("D", "N", "N", "D"), ("N", "N", "D", "N"), ("N", "N", "N", "N")]
BCS_3D = [("N", "D", "D", "D", "D", "D"), ("D", "N", "N", "D", "N", "N")]


def _dense_L(g):
    return np.stack([O.apply_L(g, e) for e in np.eye(g.size)], axis=1)


def _textbook_spectrum(g):
    """lambda^2 of every tensor mode, from the 1D formulas alone: angles
    k pi / M (two faces of one kind; k = 1..M-1 Dirichlet, 0..M Neumann) or
    (k - 1/2) pi / M (one of each), M = n + 1, symbol 4 s / h^2 or
    4 (s + s^2/3) / h^2 with s = sin^2(angle / 2)."""
    per_axis = []
    for a in range(g.dim):
        M = g.n[a] + 1
        lo, hi = g.bc[2 * a], g.bc[2 * a + 1]
        if lo == hi == "D":
            th = np.arange(1, M) * math.pi / M
        elif lo == hi == "N":
            th = np.arange(0, M + 1) * math.pi / M
        else:
            th = (np.arange(1, M + 1) - 0.5) * math.pi / M
        s = np.sin(th / 2) ** 2
        per_axis.append((4 * s if g.order == 2 else 4 * (s + s * s / 3)) / g.h[a] ** 2)
    lam2 = per_axis[0]
    for a in range(1, g.dim):
        lam2 = np.add.outer(per_axis[a], lam2).reshape(-1)
    return np.sort(lam2)


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("bc", BCS_2D + BCS_3D)
def test_dense_spectrum_is_the_tensor_cosine_sine_spectrum(order, bc):
    n = (5, 4) if len(bc) == 4 else (3, 4, 3)
    L = (1.0, 0.7) if len(bc) == 4 else (1.0, 0.8, 0.9)
    g = O.Grid(n, L, order, bc)
    A = _dense_L(g)
    ev = np.sort(-np.linalg.eigvals(A).real)
    ref = _textbook_spectrum(g)
    assert ev.shape == ref.shape
    np.testing.assert_allclose(ev, ref, rtol=0, atol=1e-12 * ref.max())
    np.testing.assert_allclose(np.sort(O.spectrum_modes(g)), ref, rtol=0, atol=1e-12 * ref.max())


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("bc", BCS_2D)
def test_modes_are_eigenvectors_pointwise(order, bc):
    g = O.Grid((9, 7), (1.0, 0.75), order, bc)
    lam2 = O.spectrum_modes(g)
    nx = g.nact[0]
    for kx, ky in [(0, 0), (1, 2), (nx - 1, 3), (4, g.nact[1] - 1)]:
        phi = O.tensor_mode(g, (kx, ky))
        l2 = lam2[ky * nx + kx]
        r = O.apply_L(g, phi) + l2 * phi
        assert np.max(np.abs(r)) <= 1e-11 * max(l2, 1.0) * np.max(np.abs(phi))
        if l2 > 0:
            assert abs(O.rayleigh_lambda(g, phi) ** 2 - l2) <= 1e-12 * l2


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("bc", BCS_2D + BCS_3D)
def test_symmetric_in_trapezoid_weights_only(order, bc):
    n = (6, 5) if len(bc) == 4 else (3, 4, 3)
    L = (1.0, 0.7) if len(bc) == 4 else (1.0, 0.8, 0.9)
    g = O.Grid(n, L, order, bc)
    A = _dense_L(g)
    WA = O.trapezoid_weights(g)[:, None] * A
    assert np.max(np.abs(WA - WA.T)) <= 1e-13 * np.max(np.abs(A))
    assert np.max(np.abs(A - A.T)) > 0.1 * np.max(np.abs(A))  # not symmetric without the weights


@pytest.mark.parametrize("order", [2, 4])
def test_constants_in_the_kernel_of_an_all_neumann_box(order):
    g = O.Grid((8, 6, 5), (1.0, 0.7, 0.6), order, ("N",) * 6)
    Lu = O.apply_L(g, np.ones(g.size))
    assert np.max(np.abs(Lu)) <= 1e-9 * np.max(np.abs(O.apply_L(g, np.arange(g.size, dtype=float))))
    # a constant is the zero mode of S's spectrum: beta_d at lambda = 0 (eq. betad)
    prm = O.filter_params(11.0, 2, 24)
    Sv = O.filter_explicit(g, prm, np.ones(g.size))
    np.testing.assert_allclose(Sv, O.beta_d(0.0, prm)[0] * np.ones(g.size), rtol=0, atol=1e-13)


def _symmetric_full(u, m, axis_len_full):
    """Full-axis vector of 2m+1 entries from its upper half u (indices m..2m),
    symmetric about index m."""
    full = np.empty(axis_len_full)
    full[m:] = u
    full[:m] = u[1:][::-1]
    return full


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("halve", ["x", "y", "xy", "x_lower"])
def test_symmetry_plane_is_the_neumann_half_box(order, halve):
    """S on the half of a Dirichlet box with a Neumann face on the symmetry
    plane equals S of the symmetric extension on the whole box, restricted
    (Section "Numerical results": the symmetry plane of the double
    ellipsoid)."""
    mx, my = 7, 5
    nxf, nyf = 2 * mx + 1, 2 * my + 1
    Lx, Ly = 1.0, 0.8
    hx, hy = Lx / (nxf + 1), Ly / (nyf + 1)
    rng = np.random.default_rng(3)
    full_g = O.Grid((nxf, nyf), (Lx, Ly), order)
    prm = O.filter_params(13.0, 2, 40)
    # half box along the chosen axes: interior m points, length (m + 1) h
    hx_half, hy_half = "x" in halve, "y" in halve
    bc = ["D", "D", "D", "D"]
    nh = [nxf, nyf]
    Lh = [Lx, Ly]
    if hx_half:
        nh[0], Lh[0] = mx, (mx + 1) * hx
        bc[0 if halve != "x_lower" else 1] = "N"
    if hy_half:
        nh[1], Lh[1] = my, (my + 1) * hy
        bc[2] = "N"
    half_g = O.Grid(tuple(nh), tuple(Lh), order, tuple(bc))
    u = rng.standard_normal(half_g.size).reshape(half_g.shape)  # (y, x)
    # symmetric extension: rows along y, columns along x
    v = u
    if hx_half:
        if halve == "x_lower":   # the half is indices 0..mx (Neumann face on its upper side)
            v = np.stack([np.concatenate([r, r[:-1][::-1]]) for r in v])
        else:
            v = np.stack([_symmetric_full(r, mx, nxf) for r in v])
    if hy_half:
        v = np.stack([_symmetric_full(c, my, nyf) for c in v.T]).T
    assert v.shape == full_g.shape
    Sv = O.filter_explicit(full_g, prm, v.reshape(-1)).reshape(full_g.shape)
    ys = slice(my, None) if hy_half else slice(None)
    xs = slice(None)
    if hx_half:
        xs = slice(0, mx + 1) if halve == "x_lower" else slice(mx, None)
    ref = Sv[ys, xs]
    got = O.filter_explicit(half_g, prm, u.reshape(-1)).reshape(half_g.shape)
    assert abs(half_g.h[0] - hx) < 1e-15 and abs(half_g.h[1] - hy) < 1e-15
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


def test_closed_form_filter_equals_dst_on_dirichlet_boxes():
    """The general mode expansion reduces to the sine transform on Dirichlet boxes."""
    g = O.Grid((9, 6), (1.0, 0.6), 4)
    v = np.random.default_rng(5).standard_normal(g.size)
    prm = O.filter_params(10.0, 1, 30)
    fn = lambda lam2: O.beta_tilde(np.sqrt(lam2), prm)
    np.testing.assert_allclose(O.modes_closed_form(g, v, fn), O.filter_closed_form(g, prm, v), atol=1e-13)


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("bc", [("N", "D", "D", "N"), ("N", "N", "N", "N")])
def test_time_stepping_equals_mode_expansion(order, bc):
    g = O.Grid((12, 9), (1.0, 0.7), order, bc)
    v = np.random.default_rng(2).standard_normal(g.size)
    prm = O.filter_params(15.0, 3, 36)
    np.testing.assert_allclose(O.filter_explicit(g, prm, v), O.filter_closed_form(g, prm, v), rtol=0,
                               atol=1e-12 * np.max(np.abs(v)))
