"""GPU parity of the double-FP32 wave-solve (EW_FP32X2: fields as pairs of FP32
numbers, about 48 significant bits, FP64 vectors in and out) against the FP64
oracle, and the mixed-precision eigen-solver whose FP64-accuracy images use it
(refine_fp64 = 3).

Tolerance: a pair operation rounds at about 2^-46 relative (measured 7.5e-15
for additions, 1.2e-14 for products); a leapfrog step makes a few of them per
point and the scheme is neutrally stable, so ||S v - S_x2 v||_2 / ||v||_2 stays
below C N_t 2^-46; C = 4 as for FP32 (measured values are far inside).
Eigenvalues after refinement: 1e-9 relative with eig-res <= 1e-8, as for
refine_fp64 = 1.
"""
import math

import numpy as np
import pytest
import torch

import ew_inputs
from oracle import oracle as O

pytestmark = pytest.mark.gpu
EPSX2 = 2.0 ** -46


@pytest.fixture(scope="module")
def ew():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_18282_gb300 as ew
    assert torch.cuda.is_available()
    return ew


def _run(ew, n, L, order, omega, bc=None, tb=0, nvec=1, Np=1, seed=7):
    g = ew.ew_grid_create(2, n, L, order=order, prec="fp32x2", bc=bc)
    p = ew.filter_params(omega, num_periods=Np, temporal_block=tb)
    info, _ = ew.ew_filter_setup(g, p)
    v = ew_inputs.uniform_pm1(seed, g.size * nvec)
    vin = torch.tensor(v, device="cuda", dtype=torch.float64)
    vout = torch.full_like(vin, float("nan"))
    ew.ew_filter_apply(g, p, vin, vout, nvec=nvec)
    torch.cuda.synchronize()
    g.close()
    return v, vout.cpu().numpy(), info


@pytest.mark.parametrize("n,L,order,bc,tb", [
    ((300, 70), (1.0, 0.7), 4, None, 0),               # tuned blocked kernel, ragged tiles
    ((300, 70), (1.0, 0.7), 4, None, 1),               # one step per launch
    ((300, 70), (1.0, 0.7), 2, None, 2),
    ((300, 70), (1.0, 0.7), 4, ("N", "D", "D", "N"), 0),  # Neumann faces: the general staging
    ((61, 40), (1.0, 0.65), 4, None, 0),               # whole grid in one CTA
    ((3, 2), (0.3, 0.6), 4, ("N", "N", "D", "N"), 0),
])
def test_parity_with_the_fp64_oracle(ew, n, L, order, bc, tb):
    v, out, info = _run(ew, n, L, order, 23.0, bc=bc, tb=tb, nvec=2)
    size = len(v) // 2
    og = O.Grid(n, L, order, bc)
    prm = O.filter_params(23.0, 1, info["steps_per_period"])
    for j in range(2):
        ref = O.filter_explicit(og, prm, v[j * size:(j + 1) * size])
        err = np.linalg.norm(out[j * size:(j + 1) * size] - ref) / np.linalg.norm(v[j * size:(j + 1) * size])
        assert err < 4 * info["Nt"] * EPSX2, (j, err)


def test_far_more_accurate_than_fp32_on_the_eigen_workload(ew):
    """One period on the full 2047 x 3071 order-4 rectangle at omega = 150 for a
    sine mode: the pair arithmetic stays within its bound of the closed form
    (the FP32 wave-solve is about 1e-6 away)."""
    n, L = (2047, 3071), (1.0, 1.5)
    og = O.Grid(n, L, 4)
    k = (140, 211)
    phi = O.sine_mode(og, k)
    lam = math.sqrt(O.lambda2_closed_form(og, [k])[0])
    g = ew.ew_grid_create(2, n, L, order=4, prec="fp32x2")
    p = ew.filter_params(150.0)
    info, _ = ew.ew_filter_setup(g, p)
    beta = O.beta_tilde(lam, O.filter_params(150.0, 1, info["steps_per_period"]))[0]
    vin = torch.tensor(phi, device="cuda")
    vout = torch.empty_like(vin)
    ew.ew_filter_apply(g, p, vin, vout)
    torch.cuda.synchronize()
    g.close()
    err = np.linalg.norm(vout.cpu().numpy() - beta * phi) / np.linalg.norm(phi)
    assert err < 4 * info["Nt"] * EPSX2, err


def test_eigs_refined_with_pair_arithmetic_images(ew):
    """refine_fp64 = 3: the FP64-accuracy images of the refinement in pair
    arithmetic; same acceptance as refine_fp64 = 1."""
    n, L, omega, Np, nw = (255, 383), (1.0, 1.5), 60.0, 64, 8
    g = ew.ew_grid_create(2, n, L, order=4, prec="fp32")
    p = ew.filter_params(omega, num_periods=Np)
    info, _ = ew.ew_filter_setup(g, p)
    e = ew.eigs_params(nw, krylov_dim=32, block=2, seed=11, refine_fp64=3, max_wave_solves=4000)
    lam, rep, st = ew.ew_arnoldi_eigs(g, p, e)
    g.close()
    og = O.Grid(n, L, 4)
    lam_all = np.sqrt(O.spectrum(og)[0])
    b = O.beta_tilde(lam_all, O.filter_params(omega, Np, info["steps_per_period"]))
    want = lam_all[np.argsort(-b)[:nw]]
    np.testing.assert_allclose(np.sort(lam), np.sort(want), rtol=1e-9)
    assert np.all(rep["eig_res"][:nw] <= 1e-8), rep["eig_res"]
    assert rep["wave_solves_fp64"] > 0


def test_other_entry_points_refuse_pair_grids(ew):
    g = ew.ew_grid_create(2, (31, 31), (1.0, 1.0), order=2, prec="fp32x2")
    x = torch.ones(g.size, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    for call in (lambda: ew.ew_apply_L(g, x, y), lambda: ew.ew_rayleigh(g, x),
                 lambda: ew.ew_arnoldi_eigs(g, ew.filter_params(10.0), ew.eigs_params(2, krylov_dim=8)),
                 lambda: ew.ew_implicit_step_mg(g, 1e-4, x, y, ew.mg_params())):
        with pytest.raises(ew.EWError, match="EW_EUNSUPPORTED"):
            call()
    g.close()
