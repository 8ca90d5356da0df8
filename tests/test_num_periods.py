"""Choice of the number of filter periods N_p (host code of the library, no
GPU): the convergence estimate of simultaneous iteration, CR = beta_{N_a+1} /
beta_{N_r} (Section "Estimating the EigenWave convergence rate based on
simultaneous iteration", eq. subSpaceIterationCR), over the box's discrete
spectrum, and the N_p minimising N_p / (-ln CR).

Pinned against the oracle: the whole closed-form spectrum of the box (every
tensor sine mode) and the oracle's closed-form filter function beta~_d (eqs.
betad, discreteExplicitLambdaTilde), an implementation independent of the
library's sum over the quadrature weights and of its windowed enumeration.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


@pytest.fixture(scope="module")
def ew():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_18282_gb300 as ew
    return ew


def _reference(n, L, order, omega, nw, na, spp, max_periods, bc=None):
    og = O.Grid(n, L, order, bc)
    lam = np.sqrt(O.spectrum_modes(og) if og.neumann else O.spectrum(og)[0])
    crs, costs = [], []
    npv = 1
    while npv <= max_periods:
        b = np.sort(O.beta_tilde(lam, O.filter_params(omega, npv, spp)))[::-1]
        cr = max(b[na], 0.0) / b[nw - 1] if b[nw - 1] > 0 else 1.0
        crs.append(cr)
        costs.append(npv / -math.log(max(cr, 1e-300)) if cr < 1 else math.inf)
        npv *= 2
    return np.array(crs), 2 ** int(np.argmin(costs))


@pytest.mark.parametrize("n,L,order,omega,nw,na", [
    ((63, 95), (1.0, 1.5), 4, 40.0, 8, 24),
    ((127, 90), (1.0, 0.7), 2, 75.0, 4, 12),
    ((15, 17, 19), (1.0, 1.1, 1.2), 2, 25.0, 6, 18),
])
def test_matches_closed_form_spectrum(ew, n, L, order, omega, nw, na):
    g = ew.ew_grid_create(len(n), n, L, order=order, prec="fp32")  # no GPU work
    p = ew.filter_params(omega)
    info, _ = ew.ew_filter_setup(g, p)
    npv, cr = ew.ew_choose_num_periods(g, p, nw, na, max_periods=64)
    ref_cr, ref_np = _reference(n, L, order, omega, nw, na, info["steps_per_period"], 64)
    np.testing.assert_allclose(cr, ref_cr, rtol=1e-8, atol=1e-12)
    assert npv == ref_np
    g.close()


@pytest.mark.parametrize("n,L,order,omega,nw,na,bc", [
    ((63, 95), (1.0, 1.5), 4, 40.0, 8, 24, ("N", "D", "D", "N")),
    ((40, 30), (1.0, 0.7), 2, 3.0, 3, 10, ("N", "N", "N", "N")),   # lambda = 0 in the spectrum
    ((15, 17, 19), (1.0, 1.1, 1.2), 2, 25.0, 6, 18, ("D", "N", "N", "D", "N", "N")),
])
def test_matches_closed_form_spectrum_with_neumann_faces(ew, n, L, order, omega, nw, na, bc):
    """Neumann faces change the per-axis mode angles (tensor cosine / mixed
    modes, one more active point per Neumann face)."""
    g = ew.ew_grid_create(len(n), n, L, order=order, prec="fp32", bc=bc)
    p = ew.filter_params(omega)
    info, _ = ew.ew_filter_setup(g, p)
    npv, cr = ew.ew_choose_num_periods(g, p, nw, na, max_periods=64)
    ref_cr, ref_np = _reference(n, L, order, omega, nw, na, info["steps_per_period"], 64, bc)
    np.testing.assert_allclose(cr, ref_cr, rtol=1e-8, atol=1e-12)
    assert npv == ref_np
    g.close()


def test_longer_filters_separate_dense_spectra(ew):
    """The paper's reading: the estimate depends on how many eigenvalues share
    the peak, so on the 2047 x 3071 rectangle at omega = 150 (about 36
    eigenvalues per unit of lambda) CR falls as N_p grows, and the chosen N_p
    is well above 1."""
    g = ew.ew_grid_create(2, (2047, 3071), (1.0, 1.5), order=4, prec="fp32")
    p = ew.filter_params(150.0)
    npv, cr = ew.ew_choose_num_periods(g, p, 8, 32, max_periods=1024)
    assert cr[-1] < cr[0] and npv >= 16
    g.close()


def test_rejects_bad_requests(ew):
    g = ew.ew_grid_create(2, (20, 20), (1.0, 1.0), order=2, prec="fp64")
    p = ew.filter_params(10.0)
    for args in [(0, 8), (8, 8), (4, 401)]:
        with pytest.raises(ew.EWError):
            ew.ew_choose_num_periods(g, p, *args, max_periods=8)
    g.close()


def test_refuses_curvilinear_grids(ew):
    """A mapped grid's spectrum has no closed form: the estimate is refused
    (host work only, no GPU)."""
    import ew_inputs
    n = (20, 15)
    g = ew.ew_grid_create_mapped(n, ew_inputs.mapped_vertices(*n, "square_warp"), prec="fp32")
    with pytest.raises(ew.EWError) as e:
        ew.ew_choose_num_periods(g, ew.filter_params(10.0), 4, 12, max_periods=8)
    assert e.value.status == 7
    g.close()
