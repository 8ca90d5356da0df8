"""GPU parity on a single curvilinear grid (the mapping method, Section
"Discrete approximations"): the library's 9-point kernels against the FP64
oracle's conservative form (ew_oracle.c: og_mapped_*), the rotated box against
the library's own box kernels, and the Krylov solver (run on
J^{1/2} S J^{-1/2}) against the oracle's dense eigenpairs.

Tolerances as for the box grids: FP64 1e-12 relative (max norm); FP32
||dS v||_2 / ||v||_2 <= 4 N_t eps32; eigenvalues FP64 1e-10, FP32 + FP64
refinement 1e-9 with eig-res <= 1e-8.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import ew_inputs
from oracle import oracle as O

pytestmark = pytest.mark.gpu
EPS32 = float(np.finfo(np.float32).eps)


@pytest.fixture(scope="module")
def ew():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_18282_gb300 as ew
    assert torch.cuda.is_available()
    return ew


def _apply(ew, n, xy, prec, omega, Np=1, nvec=1, seed=7):
    g = ew.ew_grid_create_mapped(n, xy, prec=prec)
    p = ew.filter_params(omega, num_periods=Np)
    info, _ = ew.ew_filter_setup(g, p)
    v = ew_inputs.uniform_pm1(seed, g.size * nvec)
    dt = torch.float32 if prec == "fp32" else torch.float64
    vin = torch.tensor(v, device="cuda", dtype=dt)
    vout = torch.full_like(vin, float("nan"))
    ew.ew_filter_apply(g, p, vin, vout, nvec=nvec)
    torch.cuda.synchronize()
    g.close()
    return v, vout.cpu().double().numpy(), info


@pytest.mark.parametrize("n,kind,nvec", [((150, 97), "square_warp", 1), ((61, 40), "rotated_box", 2),
                                         ((1, 1), "square_warp", 1), ((3, 2), "square_warp", 1)])
def test_fp64_parity(ew, n, kind, nvec):
    xy = ew_inputs.mapped_vertices(*n, kind, eps=0.12, theta=0.4, lx=1.0, ly=0.65)
    v, out, info = _apply(ew, n, xy, "fp64", 23.0, nvec=nvec)
    m = O.MappedGrid(n, xy)
    prm = O.filter_params(23.0, 1, info["steps_per_period"])
    size = n[0] * n[1]
    for j in range(nvec):
        ref = O.mapped_filter_explicit(m, prm, v[j * size:(j + 1) * size])
        err = np.max(np.abs(out[j * size:(j + 1) * size] - ref)) / max(np.max(np.abs(ref)), 1e-300)
        assert err < 1e-12, (j, err)


def test_fp32_parity(ew):
    n = (300, 170)
    xy = ew_inputs.mapped_vertices(*n, "square_warp", eps=0.1)
    v, out, info = _apply(ew, n, xy, "fp32", 35.0)
    ref = O.mapped_filter_explicit(O.MappedGrid(n, xy), O.filter_params(35.0, 1, info["steps_per_period"]),
                                   v.astype(np.float32).astype(np.float64))
    assert np.linalg.norm(out - ref) / np.linalg.norm(v) < 4 * info["Nt"] * EPS32


def test_rotated_box_equals_the_box_kernels(ew):
    """A rotated box has the identity metric: the mapped kernels must give
    the box kernels' wave-solve (FP64, same time step)."""
    n, L = (120, 77), (1.0, 0.6)
    xy = ew_inputs.mapped_vertices(*n, "rotated_box", theta=0.7, lx=L[0], ly=L[1])
    gm = ew.ew_grid_create_mapped(n, xy, prec="fp64")
    gb = ew.ew_grid_create(2, n, L, order=2, prec="fp64")
    p = ew.filter_params(30.0, steps_per_period=80)
    v = torch.tensor(ew_inputs.uniform_pm1(3, gm.size), device="cuda")
    a, b = torch.empty_like(v), torch.empty_like(v)
    ew.ew_filter_apply(gm, p, v, a)
    ew.ew_filter_apply(gb, p, v, b)
    torch.cuda.synchronize()
    gm.close()
    gb.close()
    assert torch.max(torch.abs(a - b)).item() < 1e-12 * torch.max(torch.abs(b)).item()


def test_apply_L_and_weighted_rayleigh(ew):
    n = (57, 43)
    xy = ew_inputs.mapped_vertices(*n, "square_warp", eps=0.15)
    m = O.MappedGrid(n, xy)
    g = ew.ew_grid_create_mapped(n, xy, prec="fp64")
    u = ew_inputs.uniform_pm1(11, g.size)
    ut = torch.tensor(u, device="cuda")
    Lu = torch.empty_like(ut)
    ew.ew_apply_L(g, ut, Lu)
    ref = O.mapped_apply_L(m, u)
    assert np.max(np.abs(Lu.cpu().numpy() - ref)) < 1e-13 * np.max(np.abs(ref))
    lam, _ = ew.ew_rayleigh(g, ut)
    assert abs(lam[0] - O.mapped_rayleigh_lambda(m, u)) < 1e-12 * lam[0]
    g.close()


def test_fp32_couplings_are_exactly_consistent(ew):
    """L 1 = 0 exactly in FP32 at every vertex whose 3 x 3 neighbourhood is
    active (the couplings are rounded to a common grid, the centre is minus
    their sum)."""
    n = (64, 48)
    g = ew.ew_grid_create_mapped(n, ew_inputs.mapped_vertices(*n, "square_warp", eps=0.13), prec="fp32")
    one = torch.ones(g.size, device="cuda")
    Lu = torch.empty_like(one)
    ew.ew_apply_L(g, one, Lu)
    torch.cuda.synchronize()
    g.close()
    assert torch.count_nonzero(Lu.reshape(n[1], n[0])[1:-1, 1:-1]).item() == 0


def _dense_wanted(m, prm, nw):
    L = np.stack([O.mapped_apply_L(m, e) for e in np.eye(m.size)], axis=1)
    lam = np.sqrt(np.sort(-np.linalg.eigvals(L).real))
    b = O.beta_tilde(lam, prm)
    return lam[np.argsort(-b)[:nw]]


def test_eigs_fp64_against_dense_eigenpairs(ew):
    n, omega, Np, nw = (47, 41), 25.0, 4, 6
    xy = ew_inputs.mapped_vertices(*n, "square_warp", eps=0.1)
    g = ew.ew_grid_create_mapped(n, xy, prec="fp64")
    p = ew.filter_params(omega, num_periods=Np)
    info, _ = ew.ew_filter_setup(g, p)
    e = ew.eigs_params(nw, krylov_dim=24, block=2, tol=1e-11, seed=5, max_wave_solves=4000)
    V = torch.zeros(g.size * nw, dtype=torch.float64, device="cuda")
    lam, rep, st = ew.ew_arnoldi_eigs(g, p, e, vecs=V)
    g.close()
    m = O.MappedGrid(n, xy)
    want = _dense_wanted(m, O.filter_params(omega, Np, info["steps_per_period"]), nw)
    np.testing.assert_allclose(np.sort(lam), np.sort(want), rtol=1e-10)
    assert np.all(rep["eig_res"][:nw] < 1e-9)
    X = V.cpu().numpy().reshape(nw, -1)
    G = (X * O.mapped_jacobian(m)) @ X.T
    assert np.max(np.abs(G - np.eye(nw))) < 1e-9  # orthonormal in the J-weighted sums


def test_eigs_fp32_refined(ew):
    n, omega, Np, nw = (47, 41), 25.0, 4, 6
    xy = ew_inputs.mapped_vertices(*n, "square_warp", eps=0.1)
    g = ew.ew_grid_create_mapped(n, xy, prec="fp32")
    p = ew.filter_params(omega, num_periods=Np)
    info, _ = ew.ew_filter_setup(g, p)
    e = ew.eigs_params(nw, krylov_dim=24, block=2, seed=5, refine_fp64=1, max_wave_solves=4000)
    lam, rep, st = ew.ew_arnoldi_eigs(g, p, e)
    g.close()
    want = _dense_wanted(O.MappedGrid(n, xy), O.filter_params(omega, Np, info["steps_per_period"]), nw)
    np.testing.assert_allclose(np.sort(lam), np.sort(want), rtol=1e-9)
    assert np.all(rep["eig_res"][:nw] <= 1e-8)


def test_batched_call_with_a_mapped_grid(ew):
    n = (90, 70)
    xy = ew_inputs.mapped_vertices(*n, "square_warp", eps=0.1)
    grids = [ew.ew_grid_create_mapped(n, xy, prec="fp64"), ew.ew_grid_create(2, (64, 200), (0.6, 1.9), order=2,
                                                                            prec="fp64")]
    params = [ew.filter_params(20.0), ew.filter_params(12.5)]
    vs = [ew_inputs.uniform_pm1(40 + q, g.size) for q, g in enumerate(grids)]
    vin = [torch.tensor(v, device="cuda") for v in vs]
    vout = [torch.full_like(x, float("nan")) for x in vin]
    ew.ew_filter_apply_batched(grids, params, vin, vout)
    torch.cuda.synchronize()
    info, _ = ew.ew_filter_setup(grids[0], params[0])
    ref = O.mapped_filter_explicit(O.MappedGrid(n, xy), O.filter_params(20.0, 1, info["steps_per_period"]), vs[0])
    assert np.max(np.abs(vout[0].cpu().numpy() - ref)) < 1e-12 * np.max(np.abs(ref))
    info, _ = ew.ew_filter_setup(grids[1], params[1])
    ref = O.filter_explicit(O.Grid((64, 200), (0.6, 1.9), 2), O.filter_params(12.5, 1, info["steps_per_period"]), vs[1])
    assert np.max(np.abs(vout[1].cpu().numpy() - ref)) < 1e-12 * np.max(np.abs(ref))
    for g in grids:
        g.close()


def test_unsupported_entry_points(ew):
    n = (31, 31)
    g = ew.ew_grid_create_mapped(n, ew_inputs.mapped_vertices(*n, "square_warp"), prec="fp64")
    x = torch.zeros(g.size, dtype=torch.float64, device="cuda")
    with pytest.raises(ew.EWError, match="EW_EUNSUPPORTED"):
        ew.ew_implicit_step_mg(g, 1e-4, torch.ones_like(x), x, ew.mg_params())
    with pytest.raises(ew.EWError, match="EW_EUNSUPPORTED"):
        ew.ew_choose_num_periods(g, ew.filter_params(10.0), 4, 12)
    p = ew.filter_params(10.0)
    st = ew._lib.lib.ew_filter_apply_noalloc(g.handle, ctypes.byref(p), ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(torch.empty_like(x).data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 7  # EW_EUNSUPPORTED
    g.close()
