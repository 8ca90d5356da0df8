"""GPU parity on boxes with Neumann faces (the paper's symmetry-plane
condition, Section "Numerical results"): the wall points are active and the
points beyond a Neumann wall are the even reflection.  Every kernel family that
reads points beyond the box is covered -- the blocked 2D kernels (each tile
and depth variant, both kernel forms), the one-CTA resident kernel, the 3D
blocked and streamed kernels, one step per launch, the batched and the
allocation-free entry points -- against the FP64 oracle; the Krylov solver
(which works with W^{1/2} S W^{-1/2}, W the trapezoid weights) against the
closed-form tensor sine / cosine spectrum.

Tolerances as in test_gpu_filter.py / test_gpu_eigs.py: FP64 1e-12 relative
(max norm); FP32 ||dS v||_2 / ||v||_2 <= 4 N_t eps32; eigenvalues FP64 1e-10,
FP32 + FP64 refinement 1e-9 with eig-res <= 1e-8.
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


def _run(ew, n, L, order, prec, omega, bc, Np=1, tb=0, nvec=1, seed=7):
    g = ew.ew_grid_create(len(n), n, L, order=order, prec=prec, bc=bc)
    p = ew.filter_params(omega, num_periods=Np, temporal_block=tb)
    info, _ = ew.ew_filter_setup(g, p)
    v = ew_inputs.uniform_pm1(seed, g.size * nvec)
    dt = torch.float32 if prec == "fp32" else torch.float64
    vin = torch.tensor(v, device="cuda", dtype=dt)
    vout = torch.full_like(vin, float("nan"))
    ew.ew_filter_apply(g, p, vin, vout, nvec=nvec)
    torch.cuda.synchronize()
    out = vout.cpu().double().numpy()
    size = g.size
    g.close()
    return v, out, info, size


def _oracle(n, L, order, omega, bc, Np, spp, v):
    return O.filter_explicit(O.Grid(n, L, order, bc), O.filter_params(omega, Np, spp), v)


BC2 = [("N", "D", "D", "N"), ("N", "N", "N", "N"), ("D", "N", "N", "D"), ("D", "D", "N", "D")]


@pytest.mark.parametrize("bc", BC2)
@pytest.mark.parametrize("n,L,order,tb", [
    ((300, 70), (1.0, 0.7), 2, 0),     # blocked kernel, 3 x 3 tiles, ragged tails
    ((300, 70), (1.0, 0.7), 4, 0),
    ((300, 70), (1.0, 0.7), 4, 3),     # another depth, ragged last block
    ((300, 70), (1.0, 0.7), 4, 1),     # one step per launch
    ((61, 40), (1.0, 0.65), 4, 0),     # whole grid resident in one CTA
    ((61, 40), (1.0, 0.65), 2, 0),
])
def test_fp64_parity_2d(ew, bc, n, L, order, tb):
    v, out, info, _ = _run(ew, n, L, order, "fp64", 23.0, bc, tb=tb)
    ref = _oracle(n, L, order, 23.0, bc, 1, info["steps_per_period"], v)
    err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
    assert err < 1e-12, err


@pytest.mark.parametrize("bc", [("N", "D", "D", "N", "N", "D"), ("N", "N", "N", "N", "N", "N")])
@pytest.mark.parametrize("order,tb", [(2, 0), (2, 3), (2, 1), (4, 0)])
def test_fp64_parity_3d(ew, bc, order, tb):
    """Order 2: the 2.5D blocked kernel (tuned and depth 3) and one step per
    launch; order 4: the z-streamed kernel.  Ragged tiles in x and y."""
    n, L = (37, 21, 13), (1.0, 0.6, 0.4)
    v, out, info, _ = _run(ew, n, L, order, "fp64", 23.0, bc, tb=tb, nvec=2)
    size = len(v) // 2
    for j in range(2):
        ref = _oracle(n, L, order, 23.0, bc, 1, info["steps_per_period"], v[j * size:(j + 1) * size])
        err = np.max(np.abs(out[j * size:(j + 1) * size] - ref)) / np.max(np.abs(ref))
        assert err < 1e-12, (j, err)


@pytest.mark.parametrize("n,bc", [((1, 1), ("N", "N", "N", "N")), ((2, 1), ("D", "N", "N", "N")),
                                  ((1, 1, 1), ("N",) * 6), ((2, 3, 1), ("N", "D", "D", "N", "N", "N"))])
@pytest.mark.parametrize("order", [2, 4])
def test_degenerate_small_grids(ew, n, bc, order):
    """Axes of three active points: the fourth-order ghosts mirror across the
    whole axis (and, in the one-CTA kernel, into the opposite ghost layer)."""
    L = tuple(0.3 * (a + 1) for a in range(len(n)))
    v, out, info, _ = _run(ew, n, L, order, "fp64", 9.0, bc, Np=2)
    ref = _oracle(n, L, order, 9.0, bc, 2, info["steps_per_period"], v)
    assert np.max(np.abs(out - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("order", [2, 4])
def test_every_tiling_variant_bit_identical(ew, order, monkeypatch):
    """Each 2D FP32 variant (tile shape, depth, shared-memory or register-
    blocked form) stages the same even-reflection ghosts and performs the same
    operations per point: bit-identical results, and within the FP32 bound of
    the oracle."""
    n, L, bc = (700, 900), (1.0, 1.3), ("N", "D", "N", "N")
    ref, count = None, 0
    for i in range(64):
        monkeypatch.setenv("EW_TB2D_VARIANT", str(i))
        try:
            v, out, info, _ = _run(ew, n, L, order, "fp32", 45.0, bc, nvec=2, seed=21)
        except ew.EWError as e:
            assert "EW_TB2D_VARIANT" in str(e)
            break
        assert np.all(np.isfinite(out))
        if ref is None:
            ref = out
        assert np.array_equal(out, ref), "variant %d differs" % i
        count += 1
    assert count >= 8
    size = len(v) // 2
    o = _oracle(n, L, order, 45.0, bc, 1, info["steps_per_period"], v[:size].astype(np.float32).astype(np.float64))
    assert np.linalg.norm(ref[:size] - o) / np.linalg.norm(v[:size]) < 4 * info["Nt"] * EPS32


@pytest.mark.parametrize("n,L,order,bc", [
    ((300, 170), (1.0, 0.6), 4, ("N", "D", "D", "N")),
    ((45, 40, 33), (1.0, 0.9, 0.8), 2, ("D", "N", "N", "D", "N", "D")),
])
def test_fp32_parity(ew, n, L, order, bc):
    v, out, info, _ = _run(ew, n, L, order, "fp32", 35.0, bc)
    ref = _oracle(n, L, order, 35.0, bc, 1, info["steps_per_period"], v.astype(np.float32).astype(np.float64))
    assert np.linalg.norm(out - ref) / np.linalg.norm(v) < 4 * info["Nt"] * EPS32


def _cosine_mode_test(ew, n, L, order, omega, bc, k, prec="fp32"):
    og = O.Grid(n, L, order, bc)
    phi = O.tensor_mode(og, k)
    lam = math.sqrt(sum(O.axis_symbol(og, a, O.axis_modes(og, a)[0][k[a]]) for a in range(len(n))))
    g = ew.ew_grid_create(len(n), n, L, order=order, prec=prec, bc=bc)
    p = ew.filter_params(omega)
    info, _ = ew.ew_filter_setup(g, p)
    beta = O.beta_tilde(lam, O.filter_params(omega, 1, info["steps_per_period"]))[0]
    dt = torch.float32 if prec == "fp32" else torch.float64
    vin = torch.tensor(phi, device="cuda", dtype=dt)
    vout = torch.empty_like(vin)
    ew.ew_filter_apply(g, p, vin, vout)
    torch.cuda.synchronize()
    out = vout.cpu().double().numpy()
    g.close()
    return np.linalg.norm(out - beta * phi) / np.linalg.norm(phi), beta, info


@pytest.mark.parametrize("k", [(0, 0), (1, 3), (140, 211), (2047, 3071)])
def test_mode_amplification_rectangle_2047x3071_symmetry_planes(ew, k):
    """Full-size 2D workload with Neumann faces at x = 0 and y = 0 (a quarter
    of a symmetric box): S phi_k = beta~_d phi_k for tensor cosine modes,
    from the quarter-wave lowest mode to the highest."""
    err, beta, info = _cosine_mode_test(ew, (2047, 3071), (1.0, 1.5), 4, 150.0, ("N", "D", "N", "D"), k)
    assert info["steps_per_period"] == 176
    assert err < 4 * info["Nt"] * EPS32, (err, beta)


def test_mode_amplification_cube_511_symmetry_plane(ew):
    """Full-size 3D workload (511^3 interior, order 2) with a Neumann face at z = 0."""
    err, beta, info = _cosine_mode_test(ew, (511, 511, 511), (1.0, 1.0, 1.0), 2, 60.0,
                                        ("D", "D", "D", "D", "N", "D"), (10, 12, 9))
    assert info["steps_per_period"] == 117
    assert err < 4 * info["Nt"] * EPS32, (err, beta)


def test_rayleigh_uses_trapezoid_weights(ew):
    n, L, bc = (40, 31), (1.0, 0.8), ("N", "N", "D", "N")
    og = O.Grid(n, L, 4, bc)
    lam2 = O.spectrum_modes(og)
    ks = [(0, 0), (3, 5), (17, 2)]
    phis = np.concatenate([O.tensor_mode(og, k) for k in ks])
    g = ew.ew_grid_create(2, n, L, order=4, prec="fp64", bc=bc)
    lam, res = ew.ew_rayleigh(g, torch.tensor(phis, device="cuda"))
    g.close()
    for j, k in enumerate(ks):
        ref = math.sqrt(lam2[k[0] + og.nact[0] * k[1]])
        assert abs(lam[j] - ref) <= 1e-12 * ref
        assert res[j] < 1e-11
    # a random vector: the weighted quotient of the oracle
    v = ew_inputs.uniform_pm1(3, og.size)
    g = ew.ew_grid_create(2, n, L, order=4, prec="fp64", bc=bc)
    lam, _ = ew.ew_rayleigh(g, torch.tensor(v, device="cuda"))
    g.close()
    assert abs(lam[0] - O.rayleigh_lambda(og, v)) <= 1e-12 * lam[0]


def _wanted(og, prm, nw):
    lam = np.sqrt(O.spectrum_modes(og))
    b = O.beta_tilde(lam, prm)
    order = np.argsort(-b)
    return lam[order[:nw]]


def test_eigs_fp64_mixed_faces(ew):
    n, L, omega, Np, nw, bc = (95, 143), (1.0, 1.5), 40.0, 2, 6, ("N", "D", "D", "N")
    g = ew.ew_grid_create(2, n, L, order=4, prec="fp64", bc=bc)
    p = ew.filter_params(omega, num_periods=Np)
    info, _ = ew.ew_filter_setup(g, p)
    e = ew.eigs_params(nw, krylov_dim=24, block=2, tol=1e-11, seed=11, max_wave_solves=4000)
    V = torch.zeros(g.size * nw, dtype=torch.float64, device="cuda")
    lam, rep, st = ew.ew_arnoldi_eigs(g, p, e, vecs=V)
    g.close()
    og = O.Grid(n, L, 4, bc)
    want = _wanted(og, O.filter_params(omega, Np, info["steps_per_period"]), nw)
    np.testing.assert_allclose(np.sort(lam), np.sort(want), rtol=1e-10)
    assert np.all(rep["eig_res"] < 1e-9)
    # eigenvectors orthonormal in the trapezoid weights, each an eigenvector of the oracle's L_h
    X = V.cpu().numpy().reshape(nw, -1)
    w = O.trapezoid_weights(og)
    G = (X * w) @ X.T
    assert np.max(np.abs(G - np.eye(nw))) < 1e-9
    for j in range(nw):
        assert O.eig_res(og, lam[j], X[j]) < 1e-9


def test_eigs_fp32_refined_symmetry_planes(ew):
    """Mixed precision on a box with two Neumann faces: FP32 Krylov stage,
    FP64 refinement to eig-res <= 1e-8, eigenvalues within 1e-9."""
    n, L, omega, Np, nw, bc = (255, 383), (1.0, 1.5), 60.0, 64, 8, ("N", "D", "N", "D")
    g = ew.ew_grid_create(2, n, L, order=4, prec="fp32", bc=bc)
    p = ew.filter_params(omega, num_periods=Np)
    info, _ = ew.ew_filter_setup(g, p)
    e = ew.eigs_params(nw, krylov_dim=32, block=2, seed=11, refine_fp64=1, max_wave_solves=4000)
    lam, rep, st = ew.ew_arnoldi_eigs(g, p, e)
    g.close()
    og = O.Grid(n, L, 4, bc)
    want = _wanted(og, O.filter_params(omega, Np, info["steps_per_period"]), nw)
    np.testing.assert_allclose(np.sort(lam), np.sort(want), rtol=1e-9)
    assert np.all(rep["eig_res"] <= 1e-8), rep["eig_res"]


def test_batched_with_neumann_boxes(ew):
    probs = [((300, 70), (1.0, 0.7), 23.0, ("N", "D", "D", "N")), ((129, 33), (1.3, 0.5), 40.0, None),
             ((64, 200), (0.6, 1.9), 12.5, ("N", "N", "N", "N"))]
    grids, params, vin, vout, vs = [], [], [], [], []
    for q, (n, L, w, bc) in enumerate(probs):
        g = ew.ew_grid_create(2, n, L, order=4, prec="fp64", bc=bc)
        v = ew_inputs.uniform_pm1(100 + q, g.size)
        grids.append(g)
        params.append(ew.filter_params(w))
        vs.append(v)
        vin.append(torch.tensor(v, dtype=torch.float64, device="cuda"))
        vout.append(torch.full_like(vin[-1], float("nan")))
    ew.ew_filter_apply_batched(grids, params, vin, vout)
    torch.cuda.synchronize()
    for q, (n, L, w, bc) in enumerate(probs):
        info, _ = ew.ew_filter_setup(grids[q], params[q])
        ref = _oracle(n, L, 4, w, bc, 1, info["steps_per_period"], vs[q])
        err = np.max(np.abs(vout[q].cpu().numpy() - ref)) / np.max(np.abs(ref))
        assert err < 1e-12, (q, err)
    for g in grids:
        g.close()


def test_noalloc_entry_point_with_neumann_faces(ew):
    n, L, bc = (300, 170), (1.0, 0.6), ("N", "D", "N", "N")
    g = ew.ew_grid_create(2, n, L, order=4, prec="fp64", bc=bc)
    p = ew.filter_params(35.0)
    info, _ = ew.ew_filter_setup(g, p)
    v = ew_inputs.uniform_pm1(9, g.size)
    vin = torch.tensor(v, device="cuda")
    out = torch.full_like(vin, float("nan"))
    st = ew._lib.lib.ew_filter_apply_noalloc(g.handle, ctypes.byref(p), ctypes.c_void_p(vin.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    g.close()
    assert st == 0
    ref = _oracle(n, L, 4, 35.0, bc, 1, info["steps_per_period"], v)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-12 * np.max(np.abs(ref))


def test_multigrid_refuses_neumann_faces(ew):
    g = ew.ew_grid_create(3, (31, 31, 31), (1.0, 1.0, 1.0), order=2, prec="fp64", bc=("N",) + ("D",) * 5)
    x = torch.zeros(g.size, dtype=torch.float64, device="cuda")
    b = torch.ones_like(x)
    with pytest.raises(ew.EWError, match="EW_EUNSUPPORTED"):
        ew.ew_implicit_step_mg(g, 1e-4, b, x, ew.mg_params())
    g.close()
