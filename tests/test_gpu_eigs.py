"""GPU eigen-solver (row a7, a8): block Krylov-Schur on S with the CUDA
wave-solve, checked against the closed-form discrete spectrum and against the
oracle's own Krylov-Schur.

Tolerances: FP64 wave-solves, eigenvalues to 1e-10 relative (Ritz residual
tol 1e-11 gives eigenvector errors ~1e-11/gap and Rayleigh-quotient errors of
their square); the FP32 path after FP64 refinement to 1e-9 relative and
eig-res <= 1e-8 (the target); FP32 first-stage eigenvalues to 1e-6 relative.
"""
import math

import numpy as np
import pytest
import torch

import ew_inputs
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ew():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_18282_gb300 as ew
    return ew


def _wanted(og, prm, nw, scheme="explicit"):
    lam = np.sqrt(O.spectrum(og)[0])
    b = O.beta_tilde(lam, prm, scheme)
    order = np.argsort(-b)
    return lam[order[:nw]], b[order[:nw]], b[order[nw]]


def _solve(ew, n, L, order, prec, omega, Np, nw, block, kdim, tol=0.0, refine=False, seed=11, vecs=False):
    g = ew.ew_grid_create(len(n), n, L, order=order, prec=prec)
    p = ew.filter_params(omega, num_periods=Np)
    info, _ = ew.ew_filter_setup(g, p)
    e = ew.eigs_params(nw, krylov_dim=kdim, block=block, tol=tol, seed=seed, refine_fp64=refine,
                       max_wave_solves=4000)
    V = torch.zeros(g.size * nw, dtype=torch.float64, device="cuda") if vecs else None
    lam, rep, st = ew.ew_arnoldi_eigs(g, p, e, vecs=V)
    g.close()
    return lam, rep, info, V


def test_fp64_rectangle_order4(ew):
    n, L, omega, Np, nw = (95, 143), (1.0, 1.5), 40.0, 2, 6
    lam, rep, info, _ = _solve(ew, n, L, 4, "fp64", omega, Np, nw, 2, 24, tol=1e-11)
    og = O.Grid(n, L, 4)
    want, beta, _ = _wanted(og, O.filter_params(omega, Np, info["steps_per_period"]), nw)
    np.testing.assert_allclose(np.sort(lam), np.sort(want), rtol=1e-10)
    np.testing.assert_allclose(np.sort(rep["beta"]), np.sort(beta), atol=1e-10)
    assert np.all(rep["eig_res"] < 1e-9)
    assert rep["n_converged"] == nw


@pytest.mark.parametrize("refine", [1, 2])
def test_fp32_with_fp64_refinement(ew, refine):
    """Mixed precision: FP32 filter steps, FP64 refinement.  Every eigenvalue
    is within 1e-9 of the closed form after refinement and within 1e-6 before;
    the FP64 stage reaches eig-res <= 1e-8.  N_p = 64 narrows the filter peak
    to about omega / N_p ~ 1, i.e. about the Krylov dimension in eigenvalues."""
    n, L, omega, Np, nw = (255, 383), (1.0, 1.5), 60.0, 64, 8
    lam, rep, info, V = _solve(ew, n, L, 4, "fp32", omega, Np, nw, 2, 32, refine=refine, vecs=True)
    og = O.Grid(n, L, 4)
    want, _, _ = _wanted(og, O.filter_params(omega, Np, info["steps_per_period"]), nw)
    np.testing.assert_allclose(np.sort(lam), np.sort(want), rtol=1e-9)
    np.testing.assert_allclose(np.sort(rep["lambda_stage1"]), np.sort(want), rtol=1e-6)
    assert np.all(rep["eig_res"] <= 1e-8), rep["eig_res"]
    assert rep["wave_solves_fp64"] > 0
    # eigenvectors: unit norm and each inside its closed-form eigenspace
    X = V.cpu().numpy().reshape(nw, -1)
    lam_all, k_all = O.spectrum(og)
    lam_all = np.sqrt(lam_all)
    for j in range(nw):
        assert abs(np.linalg.norm(X[j]) - 1.0) < 1e-10
        same = np.nonzero(np.abs(lam_all - lam[j]) < 1e-7 * lam[j])[0]
        basis = np.column_stack([O.sine_mode(og, k_all[i]) for i in same])
        assert O.eigenspace_distance(X[j], basis) < 1e-7


def test_cube_multiplicity(ew):
    """Unit cube: eigenvalues of multiplicity 3 and 6; a block of 6 finds every
    copy (the paper's tables list all of them)."""
    n, L = (15, 15, 15), (1.0, 1.0, 1.0)
    og = O.Grid(n, L, 2)
    lam_all = np.sqrt(O.spectrum(og)[0])
    # target the (1,2,3) level: six permutations
    target = math.sqrt(O.lambda2_closed_form(og, [(1, 2, 3)])[0])
    lam, rep, info, _ = _solve(ew, n, L, 2, "fp64", target, 3, 6, 6, 36, tol=1e-10)
    assert np.all(np.abs(lam - target) < 1e-9 * target), lam
    assert np.sum(np.abs(lam_all - target) < 1e-9 * target) == 6


def test_matches_oracle_krylov_schur(ew):
    """The CUDA solver and the oracle's numpy Krylov-Schur, same problem, same
    wanted set: identical eigenvalues."""
    n, L, omega, Np, nw = (47, 31), (1.2, 0.8), 30.0, 2, 5
    lam, rep, info, _ = _solve(ew, n, L, 2, "fp64", omega, Np, nw, 1, 16, tol=1e-11)
    og = O.Grid(n, L, 2)
    prm = O.filter_params(omega, Np, info["steps_per_period"])
    v0 = ew_inputs.start_block(5, og.size, 1)
    theta, X, _ = O.krylov_schur_eigs(lambda v: O.filter_explicit(og, prm, v), v0, nw, 16, tol=1e-11)
    lam_o = np.sort([O.rayleigh_lambda(og, X[:, j]) for j in range(X.shape[1])])
    np.testing.assert_allclose(np.sort(lam), lam_o, rtol=1e-10)
    np.testing.assert_allclose(np.sort(rep["beta"]), np.sort(theta), atol=1e-10)


def test_seeded_start_block_matches_host_generator(ew):
    """The library's SplitMix64 start block equals ew_inputs' (same published
    generator on both sides): passing it explicitly gives the same result."""
    n, L = (40, 30), (1.0, 0.75)
    g = ew.ew_grid_create(2, n, L, order=2, prec="fp64")
    p = ew.filter_params(25.0, num_periods=2)
    e = ew.eigs_params(3, krylov_dim=8, block=2, tol=1e-10, seed=1234)
    lam_a, _, _ = ew.ew_arnoldi_eigs(g, p, e)
    start = ew_inputs.uniform_pm1(1234, g.size * 2)
    lam_b, _, _ = ew.ew_arnoldi_eigs(g, p, e, start=torch.tensor(start, device="cuda"))
    np.testing.assert_array_equal(lam_a, lam_b)
    g.close()


def test_invalid_eigs_params(ew):
    g = ew.ew_grid_create(2, (20, 20), (1, 1), prec="fp64")
    p = ew.filter_params(10.0)
    for e in [ew.eigs_params(0), ew.eigs_params(4, krylov_dim=4, block=2), ew.eigs_params(3, block=17)]:
        with pytest.raises(ew.EWError) as ex:
            ew.ew_arnoldi_eigs(g, p, e)
        assert ex.value.status == 1
    g.close()


def _batched_box_plan(b):
    """N_p for a box of the batched workload: about 12 eigenvalues within
    omega / N_p of omega (density A omega / (2 pi) near omega)."""
    area = b["length"][0] * b["length"][1]
    return max(4, math.ceil(area * b["omega"] ** 2 / (12 * math.pi)))


def test_batched_boxes_per_problem_eigenvalues(ew):
    """Batched workload (64 uneven boxes, order 2, anisotropic h): the 4
    eigenpairs nearest each box's omega from FP32 wave-solves with FP64
    refinement, each eigenvalue against the closed form of its own box.  Run on
    the six boxes whose eigen-solve is cheapest (the whole set costs minutes of
    GPU time; every box shares the same code path)."""
    boxes = ew_inputs.batched_boxes(ew_inputs.BASE_SEED + 3)

    def cost(b):
        hx, hy = (b["length"][a] / (b["n"][a] + 1) for a in range(2))
        spp = math.ceil((2 * math.pi / b["omega"]) / (0.8 * 2 / math.sqrt(4 / hx ** 2 + 4 / hy ** 2)))
        return b["n"][0] * b["n"][1] * spp * _batched_box_plan(b)

    for b in sorted(boxes, key=cost)[:6]:
        n, L, omega, Np = tuple(b["n"]), tuple(b["length"]), b["omega"], _batched_box_plan(b)
        lam, rep, info, _ = _solve(ew, n, L, 2, "fp32", omega, Np, 4, 2, 16, refine=1, seed=5)
        og = O.Grid(n, L, 2)
        want, _, _ = _wanted(og, O.filter_params(omega, Np, info["steps_per_period"]), 4)
        np.testing.assert_allclose(np.sort(lam), np.sort(want), rtol=1e-9)
        assert np.all(rep["eig_res"] <= 1e-8), (n, omega, rep["eig_res"])


def test_batched_eigen_solver_on_box_subset(ew):
    """The batched eigen-solver (ew_arnoldi_eigs_batched) on eight boxes of the
    64-box workload: every box's solver runs on its own thread and stream, and
    their filter applications are gathered into batched calls.  Each box's 4
    eigenvalues nearest its omega (FP32 first stage, refinement with FP64 images)
    match its own closed form to 1e-9 with eig-res <= 1e-8, and equal those of
    the one-problem solver on the same box and seed (the batched wave-solve is
    bit-identical to the single one, so the Krylov iterations coincide)."""
    boxes = ew_inputs.batched_boxes(ew_inputs.BASE_SEED + 3)

    def cost(b):
        hx, hy = (b["length"][a] / (b["n"][a] + 1) for a in range(2))
        spp = math.ceil((2 * math.pi / b["omega"]) / (0.8 * 2 / math.sqrt(4 / hx ** 2 + 4 / hy ** 2)))
        return b["n"][0] * b["n"][1] * spp * _batched_box_plan(b)

    sel = sorted(boxes, key=cost)[:8]
    grids, params, eigs = [], [], []
    for q, b in enumerate(sel):
        g = ew.ew_grid_create(2, tuple(b["n"]), tuple(b["length"]), order=2, prec="fp32")
        grids.append(g)
        params.append(ew.filter_params(b["omega"], num_periods=_batched_box_plan(b)))
        eigs.append(ew.eigs_params(4, krylov_dim=16, block=2, seed=5 + q, refine_fp64=1, max_wave_solves=4000))
    lams, reps, sts, rounds = ew.ew_arnoldi_eigs_batched(grids, params, eigs)
    assert all(s == 0 for s in sts), sts
    assert rounds >= 1
    for q, b in enumerate(sel):
        n, L = tuple(b["n"]), tuple(b["length"])
        info, _ = ew.ew_filter_setup(grids[q], params[q])
        og = O.Grid(n, L, 2)
        want, _, _ = _wanted(og, O.filter_params(b["omega"], _batched_box_plan(b), info["steps_per_period"]), 4)
        np.testing.assert_allclose(np.sort(lams[q]), np.sort(want), rtol=1e-9)
        assert np.all(reps[q]["eig_res"] <= 1e-8), (q, reps[q]["eig_res"])
        lam1, rep1, _ = ew.ew_arnoldi_eigs(grids[q], params[q], eigs[q])
        np.testing.assert_allclose(lams[q], lam1, rtol=1e-12, atol=0)
        assert rep1["wave_solves"] == reps[q]["wave_solves"]
    for g in grids:
        g.close()


def test_rectangle_2047x3071_eight_pairs_full_size(ew):
    """The 2047 x 3071 order-4 workload at full size: the 8 eigenpairs nearest
    omega = 150 from FP32 wave-solves (Krylov dimension 32, block 4, N_p from
    the simultaneous-iteration estimate) refined with images in double-FP32
    pairs.  Each eigenvalue matches the closed form of the box to 1e-9 and every
    eig-res is <= 1e-8 (the target; about two minutes on one GPU)."""
    n, L, omega = (2047, 3071), (1.0, 1.5), 150.0
    g = ew.ew_grid_create(2, n, L, order=4, prec="fp32")
    Np, cr = ew.ew_choose_num_periods(g, ew.filter_params(omega), 8, 32, max_periods=1024)
    p = ew.filter_params(omega, num_periods=Np)
    e = ew.eigs_params(8, krylov_dim=32, block=4, seed=7, refine_fp64=3, max_wave_solves=600)
    lam, rep, st = ew.ew_arnoldi_eigs(g, p, e)
    g.close()
    # closed form: per-axis order-4 symbols with the odd-reflection closure
    per_axis = []
    for nd, ld in zip(n, L):
        h = ld / (nd + 1)
        s = np.sin(np.arange(1, nd + 1) * np.pi / (2 * (nd + 1))) ** 2
        per_axis.append(4.0 / h ** 2 * (s + s * s / 3.0))
    lam2 = per_axis[0][:, None] + per_axis[1][None, :]
    near = np.sqrt(lam2[np.abs(np.sqrt(lam2) - omega) < 2.0])
    for x in lam:
        assert np.min(np.abs(near - x)) <= 1e-9 * x, x
    assert np.all(rep["eig_res"] <= 1e-8), rep["eig_res"]
    assert len(set(np.round(lam, 9))) == 8  # eight distinct pairs (the levels are simple here)


def test_locking_keeps_the_converged_pairs(ew):
    """Krylov-Schur with locking of converged pairs (eigs.lock): the same eigenvalues
    as without it (closed form of the box, FP64), in no more wave-solves than
    twice as many (locking only changes which restart directions are kept)."""
    n, L, omega = (127, 127), (1.0, 1.0), 12.0
    og = O.Grid(n, L, 2)
    res = {}
    for lock in (False, True):
        g = ew.ew_grid_create(2, n, L, order=2, prec="fp64")
        p = ew.filter_params(omega, num_periods=2)
        info, _ = ew.ew_filter_setup(g, p)
        e = ew.eigs_params(16, krylov_dim=34, block=2, tol=1e-11, seed=3, max_wave_solves=2000, lock=lock)
        lam, rep, st = ew.ew_arnoldi_eigs(g, p, e)
        g.close()
        res[lock] = (np.sort(lam), rep)
    want, _, _ = _wanted(og, O.filter_params(omega, 2, info["steps_per_period"]), 16)
    for lock in (False, True):
        np.testing.assert_allclose(res[lock][0], np.sort(want), rtol=1e-10)
    assert res[True][1]["wave_solves"] <= 2 * res[False][1]["wave_solves"]
