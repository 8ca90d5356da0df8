"""GPU parity of the explicit wave-solve (rows a1-a5) against the FP64 oracle.

Tolerances:
  FP64: max-norm error <= 1e-12 relative to max |S v| (the target's FP64
  bound; rounding-order differences grow like N_t * 1e-16).
  FP32: a leapfrog step makes about four roundings of size eps32 |u| and the
  scheme is neutrally stable, so the error of W^n grows at most linearly in
  n; the filter weights sum to O(1), so ||S v - S_32 v|| / ||v|| stays below
  C * N_t * eps32.  C = 4 is used for the 2-norm bound.  Element by element
  the same argument applies to one point's roundings (each at most a few
  eps32 max |W^n| <= eps32 max |v| per step, carried by a propagator that is
  bounded in the max norm over one period), so every point is also checked
  against 4 N_t eps32 max |v|; the measured worst point sits about 10x inside.
"""
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


def _run(ew, n, length, order, prec, omega, Np=1, tb=0, spp=0, nvec=1, seed=7):
    dim = len(n)
    g = ew.ew_grid_create(dim, n, length, order=order, prec=prec)
    p = ew.filter_params(omega, num_periods=Np, steps_per_period=spp, temporal_block=tb)
    info, _ = ew.ew_filter_setup(g, p)
    size = int(np.prod(n))
    v = ew_inputs.uniform_pm1(seed, size * nvec)
    dt = torch.float32 if prec == "fp32" else torch.float64
    vin = torch.tensor(v, device="cuda", dtype=dt)
    vout = torch.full_like(vin, float("nan"))
    ew.ew_filter_apply(g, p, vin, vout, nvec=nvec)
    torch.cuda.synchronize()
    out = vout.cpu().double().numpy()
    g.close()
    return v, out, info


def _oracle(n, length, order, omega, Np, spp, v):
    og = O.Grid(n, length, order)
    prm = O.filter_params(omega, Np, spp)
    return O.filter_explicit(og, prm, v)


@pytest.mark.parametrize("n,length,order,tb", [
    ((300, 70), (1.0, 0.7), 2, 0),     # blocked kernel, 3 x 3 tiles, ragged tails
    ((300, 70), (1.0, 0.7), 4, 0),
    ((300, 70), (1.0, 0.7), 4, 3),     # another temporal depth, ragged last block
    ((300, 70), (1.0, 0.7), 4, 1),     # one step per launch
    ((129, 33), (1.3, 0.5), 2, 2),
    ((63, 63), (1.0, 1.0), 2, 0),      # whole grid resident in one CTA
    ((20, 9), (1.0, 0.45), 4, 0),
    ((37, 21, 13), (1.0, 0.6, 0.4), 2, 0),
    ((37, 21, 13), (1.0, 0.6, 0.4), 4, 0),
])
def test_fp64_parity(ew, n, length, order, tb):
    omega = 23.0
    v, out, info = _run(ew, n, length, order, "fp64", omega, Np=1, tb=tb)
    ref = _oracle(n, length, order, omega, 1, info["steps_per_period"], v)
    err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
    assert err < 1e-12, err


@pytest.mark.parametrize("n", [(1, 1), (1, 7), (5, 2), (3, 3, 1), (1, 1, 1), (2, 3, 4)])
@pytest.mark.parametrize("order", [2, 4])
def test_degenerate_small_grids(ew, n, order):
    length = tuple(0.3 * (a + 1) for a in range(len(n)))
    v, out, info = _run(ew, n, length, order, "fp64", 9.0, Np=2)
    ref = _oracle(n, length, order, 9.0, 2, info["steps_per_period"], v)
    assert np.max(np.abs(out - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_tiling_variants_bit_identical(ew):
    """Every tile shape and temporal depth performs the same operations per
    point, so the tuned default and fixed depths 2 and 3 agree bit for bit."""
    v, a, _ = _run(ew, (300, 140), (1.0, 0.5), 4, "fp32", 40.0, Np=2, tb=0)
    _, b, _ = _run(ew, (300, 140), (1.0, 0.5), 4, "fp32", 40.0, Np=2, tb=2)
    _, c, _ = _run(ew, (300, 140), (1.0, 0.5), 4, "fp32", 40.0, Np=2, tb=3)
    assert np.array_equal(a, b) and np.array_equal(a, c)


@pytest.mark.parametrize("order", [2, 4])
def test_every_tiling_variant_bit_identical(ew, order, monkeypatch):
    """Every 2D FP32 variant -- tile shape, temporal depth, and kernel form
    (shared-memory tiles or the register-blocked persistent kernel with bulk
    row copies) -- performs the same operations per point, so forcing each in
    turn gives the same result bit for bit.  700 x 900 with 3 vectors spans
    more tiles than SMs (persistent CTAs walk several tiles) with ragged tiles
    on two sides."""
    n, L = (700, 900), (1.0, 1.3)
    ref, count = None, 0
    for i in range(64):
        monkeypatch.setenv("EW_TB2D_VARIANT", str(i))
        try:
            _, out, _ = _run(ew, n, L, order, "fp32", 45.0, nvec=3, seed=21)
        except ew.EWError as e:  # past the end of the list
            assert "EW_TB2D_VARIANT" in str(e)
            break
        assert np.all(np.isfinite(out))
        if ref is None:
            ref = out
        assert np.array_equal(out, ref), "variant %d differs" % i
        count += 1
    assert count >= 8


def test_fp64_blocked_equals_simple(ew):
    """Temporal blocking changes only rounding order: depth 4 vs depth 1."""
    v, a, _ = _run(ew, (300, 140), (1.0, 0.5), 4, "fp64", 40.0, Np=2, tb=4)
    _, b, _ = _run(ew, (300, 140), (1.0, 0.5), 4, "fp64", 40.0, Np=2, tb=1)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(b))


@pytest.mark.parametrize("tb", [0, 2, 3])
def test_fp64_3d_blocked_equals_simple(ew, tb):
    """3D second-order temporal blocking (2.5D, levels pipelined along z)
    changes only rounding order: depths 4 (default), 2 and 3 against one step
    per launch, two vectors, ragged tiles in x and y, N_t not a multiple of
    the depth."""
    n, L = (61, 50, 23), (1.0, 0.8, 0.4)
    v, a, info = _run(ew, n, L, 2, "fp64", 30.0, Np=2, tb=tb, nvec=2)
    _, b, _ = _run(ew, n, L, 2, "fp64", 30.0, Np=2, tb=1, nvec=2)
    assert info["Nt"] % 4 != 0 or info["Nt"] % 3 != 0
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(b))


@pytest.mark.parametrize("tb", [0, 2, 3, 4])
def test_fp32_3d_blocked_equals_simple(ew, tb):
    """FP32 3D temporal blocking (each thread two adjacent columns in paired
    FP32 instructions) against one step per launch: the same operations per
    point, two vectors, ragged tiles in x and y, odd x extents (column pairs
    that straddle the box edge), the last launch shallower than the depth."""
    n, L = (61, 51, 23), (1.0, 0.8, 0.4)
    v, a, info = _run(ew, n, L, 2, "fp32", 30.0, Np=2, tb=tb, nvec=2)
    _, b, _ = _run(ew, n, L, 2, "fp32", 30.0, Np=2, tb=1, nvec=2)
    assert info["Nt"] % 4 != 0 or info["Nt"] % 3 != 0
    assert np.max(np.abs(a - b)) <= 4 * info["Nt"] * EPS32 * np.max(np.abs(v))


@pytest.mark.parametrize("nvec,chunk,prec", [(16, 0, "fp32"), (5, 2, "fp32"), (7, 3, "fp64"), (2, 0, "fp32")])
def test_host_buffers_equal_device_path(ew, nvec, chunk, prec):
    """ew_filter_apply_host (vectors in host memory, chunked copies overlapped
    with the wave-solves) gives the bits of ew_filter_apply on the same vectors,
    from pinned and from pageable host buffers; a ragged last chunk."""
    n, L = (300, 170), (1.0, 0.6)
    g = ew.ew_grid_create(2, n, L, order=4, prec=prec)
    p = ew.filter_params(35.0)
    dt = torch.float32 if prec == "fp32" else torch.float64
    v = torch.tensor(ew_inputs.uniform_pm1(31, g.size * nvec), dtype=dt)
    h_in = v.pin_memory()
    h_out = torch.full_like(v, float("nan")).pin_memory()
    ew.ew_filter_apply_host(g, p, h_in, h_out, nvec=nvec, chunk=chunk)
    torch.cuda.synchronize()
    d_out = torch.empty(g.size * nvec, dtype=dt, device="cuda")
    ew.ew_filter_apply(g, p, v.cuda(), d_out, nvec=nvec)
    torch.cuda.synchronize()
    assert torch.equal(h_out, d_out.cpu())
    h_page = torch.full_like(v, float("nan"))
    ew.ew_filter_apply_host(g, p, v, h_page, nvec=nvec, chunk=chunk)
    torch.cuda.synchronize()
    assert torch.equal(h_page, h_out)
    with pytest.raises(ew.EWError, match="EW_EINVAL"):
        ew.ew_filter_apply_host(g, p, h_in, h_out, nvec=nvec, chunk=-1)
    g.close()


def test_multi_vector_block(ew):
    """nvec vectors in one call equal separate calls, bit for bit."""
    n, L = (150, 40), (1.0, 0.3)
    v3, out3, _ = _run(ew, n, L, 4, "fp32", 31.0, nvec=3, seed=5)
    size = n[0] * n[1]
    for j in range(3):
        g = ew.ew_grid_create(2, n, L, order=4, prec="fp32")
        p = ew.filter_params(31.0)
        vin = torch.tensor(v3[j * size:(j + 1) * size], device="cuda", dtype=torch.float32)
        vout = torch.empty_like(vin)
        ew.ew_filter_apply(g, p, vin, vout)
        torch.cuda.synchronize()
        assert np.array_equal(vout.cpu().double().numpy(), out3[j * size:(j + 1) * size])
        g.close()


@pytest.mark.parametrize("n,length,order,tb", [
    ((300, 170), (1.0, 0.6), 4, 0),
    ((300, 170), (1.0, 0.6), 2, 0),
    ((45, 40, 33), (1.0, 0.9, 0.8), 2, 0),
])
def test_fp32_parity(ew, n, length, order, tb):
    omega = 35.0
    v, out, info = _run(ew, n, length, order, "fp32", omega, Np=1, tb=tb)
    ref = _oracle(n, length, order, omega, 1, info["steps_per_period"], v.astype(np.float32).astype(np.float64))
    rel2 = np.linalg.norm(out - ref) / np.linalg.norm(v)
    assert rel2 < 4 * info["Nt"] * EPS32, (rel2, info["Nt"])
    relmax = np.max(np.abs(out - ref)) / np.max(np.abs(v))
    assert relmax < 4 * info["Nt"] * EPS32, (relmax, info["Nt"])


def _mode_test(ew, n, length, order, omega, k, prec="fp32"):
    dim = len(n)
    og = O.Grid(n, length, order)
    phi = O.sine_mode(og, k)
    lam = math.sqrt(O.lambda2_closed_form(og, [k])[0])
    g = ew.ew_grid_create(dim, n, length, order=order, prec=prec)
    p = ew.filter_params(omega)
    info, _ = ew.ew_filter_setup(g, p)
    prm = O.filter_params(omega, 1, info["steps_per_period"])
    beta = O.beta_tilde(lam, prm)[0]
    dt = torch.float32 if prec == "fp32" else torch.float64
    vin = torch.tensor(phi, device="cuda", dtype=dt)
    vout = torch.empty_like(vin)
    ew.ew_filter_apply(g, p, vin, vout)
    torch.cuda.synchronize()
    out = vout.cpu().double().numpy()
    g.close()
    err = np.linalg.norm(out - beta * phi) / np.linalg.norm(phi)
    return err, beta, info


@pytest.mark.parametrize("k", [(1, 1), (137, 210), (2047, 3071)])
def test_mode_amplification_rectangle_2047x3071_order4(ew, k):
    """Full-size 2D workload (unit width x 1.5, order 4): S phi_k = beta~_d phi_k."""
    err, beta, info = _mode_test(ew, (2047, 3071), (1.0, 1.5), 4, 150.0, k)
    assert info["steps_per_period"] == 176
    assert err < 4 * info["Nt"] * EPS32, (err, beta)


def test_mode_amplification_cube_511_order2(ew):
    """Full-size 3D workload (511^3, order 2): S phi_k = beta~_d phi_k."""
    err, beta, info = _mode_test(ew, (511, 511, 511), (1.0, 1.0, 1.0), 2, 60.0, (11, 13, 9))
    assert info["steps_per_period"] == 117
    assert err < 4 * info["Nt"] * EPS32, (err, beta)


def test_full_size_random_parity_rectangle(ew):
    """Full-size 2D workload on a seeded uniform[-1,1] start vector, one
    period, FP32 GPU vs the FP64 oracle (the oracle takes seconds here)."""
    n, L, omega = (2047, 3071), (1.0, 1.5), 150.0
    v, out, info = _run(ew, n, L, 4, "fp32", omega, Np=1, seed=ew_inputs.BASE_SEED + 1)
    ref = _oracle(n, L, 4, omega, 1, info["steps_per_period"], v.astype(np.float32).astype(np.float64))
    rel2 = np.linalg.norm(out - ref) / np.linalg.norm(v)
    assert rel2 < 4 * info["Nt"] * EPS32, rel2
    # every point (max norm), the corners and seams of the tiling included
    relmax = np.max(np.abs(out - ref)) / np.max(np.abs(v))
    assert relmax < 4 * info["Nt"] * EPS32, relmax


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_stencil_coefficients_exactly_consistent(ew, order, prec):
    """The stored stencil coefficients sum to exactly zero, so L_h applied to
    the constant 1 is exactly 0 away from the boundary.  Coefficients rounded
    one by one would leave a mass term of about eps |c0|: in FP32 on fine grids
    a frequency error of up to 1e-2 for the low modes."""
    n, L = (2047, 301), (1.0, 0.147)
    g = ew.ew_grid_create(2, n, L, order=order, prec=prec)
    dt = torch.float32 if prec == "fp32" else torch.float64
    x = torch.ones(n[0] * n[1], dtype=dt, device="cuda")
    y = torch.empty_like(x)
    ew.ew_apply_L(g, x, y)
    torch.cuda.synchronize()
    Y = y.cpu().numpy().reshape(n[1], n[0])
    assert np.all(Y[2:-2, 2:-2] == 0.0)
    g.close()


def test_apply_L_and_rayleigh(ew):
    n, L = (70, 50, 30), (1.0, 0.8, 0.5)
    og = O.Grid(n, L, 4)
    g = ew.ew_grid_create(3, n, L, order=4, prec="fp64")
    u = ew_inputs.uniform_pm1(3, og.size)
    ut = torch.tensor(u, device="cuda")
    Lu = torch.empty_like(ut)
    ew.ew_apply_L(g, ut, Lu)
    torch.cuda.synchronize()
    ref = O.apply_L(og, u)
    assert np.max(np.abs(Lu.cpu().numpy() - ref)) < 1e-12 * np.max(np.abs(ref))
    k = (3, 5, 2)
    phi = np.stack([O.sine_mode(og, k), u])
    lam, res = ew.ew_rayleigh(g, torch.tensor(phi.reshape(-1), device="cuda"), nvec=2)
    assert abs(lam[0] - math.sqrt(O.lambda2_closed_form(og, [k])[0])) < 1e-12 * lam[0]
    assert res[0] < 1e-12
    assert abs(lam[1] - O.rayleigh_lambda(og, u)) < 1e-12 * lam[1]
    assert abs(res[1] - O.eig_res(og, O.rayleigh_lambda(og, u), u)) < 1e-10 * res[1]
    g.close()


def test_power_iteration_unit_square_63(ew):
    """Unit square 63x63, order 2, FP64 explicit at CFL 0.8, omega = 20, 40
    power iterations (Algorithm EigenWave) from a seeded start vector: the
    iterate equals the closed form S^40 v / ||S^40 v|| to 1e-12, and the
    Rayleigh quotient equals the oracle's on that vector."""
    n, L, omega = (63, 63), (1.0, 1.0), 20.0
    og = O.Grid(n, L, 2)
    g = ew.ew_grid_create(2, n, L, order=2, prec="fp64")
    p = ew.filter_params(omega)
    info, _ = ew.ew_filter_setup(g, p)
    assert info["steps_per_period"] == 36
    v0 = ew_inputs.uniform_pm1(ew_inputs.BASE_SEED, og.size)
    v = torch.tensor(v0, device="cuda")
    betas, done, lam = ew.ew_power_iteration(g, p, v, 40)
    assert done == 40
    prm = O.filter_params(omega, 1, 36)
    ref = O.filter_closed_form(og, prm, v0 / np.linalg.norm(v0), 40)
    ref /= np.linalg.norm(ref)
    got = v.cpu().numpy()
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    assert abs(lam - O.rayleigh_lambda(og, ref)) < 1e-12 * lam
    # the two closed-form levels nearest omega (both double) bound the estimate
    lam_all = np.sqrt(O.spectrum(og)[0])
    b = O.beta_tilde(lam_all, prm)
    top = lam_all[np.argsort(-b)[:4]]
    assert top.min() - 1e-9 <= lam <= top.max() + 1e-9
    # beta of the last iteration is (S v_39, v_39) for the closed-form v_39
    v39 = O.filter_closed_form(og, prm, v0 / np.linalg.norm(v0), 39)
    v39 /= np.linalg.norm(v39)
    beta_ref = float(np.dot(O.filter_closed_form(og, prm, v39, 1), v39))
    assert abs(betas[-1] - beta_ref) < 1e-12
    g.close()


def test_invalid_calls(ew):
    g = ew.ew_grid_create(2, (40, 30), (1, 1), prec="fp32")
    p = ew.filter_params(10.0)
    x = torch.zeros(2 * 1200, device="cuda")
    with pytest.raises(ew.EWError) as e:
        ew.ew_filter_apply(g, p, x[:1200], x[600:1800])
    assert e.value.status == 1
    with pytest.raises(ew.EWError):
        ew.ew_filter_apply(g, p, x[:1200], x[1200:], nvec=0)
    with pytest.raises(TypeError):
        ew.ew_filter_apply(g, p, x[:1200].double(), x[1200:].double())
    g.close()


@pytest.mark.parametrize("form", ["rb:0", "tma:0"])
def test_staging_wait_gives_up_cleanly(ew, form, monkeypatch):
    """Failure handling without a fault: the waits of the register-blocked
    (rb) and TMA-staged (tma) forms on their asynchronous copies are bounded
    (about 2 s).  A test hook makes every CTA expect 16 bytes that never
    arrive, so its first wait runs out; the kernel records that and returns,
    the next synchronising call reports EW_ETIMEOUT, and the device stays
    usable: the same wave-solve without the hook then matches the
    shared-memory kernel bit for bit."""
    n, L = (300, 140), (1.0, 0.5)
    g = ew.ew_grid_create(2, n, L, order=4, prec="fp32")
    p = ew.filter_params(400.0, num_periods=1)  # about 10 steps: a few launches, each wait runs out once
    vin = torch.tensor(ew_inputs.uniform_pm1(77, g.size), dtype=torch.float32, device="cuda")
    out = torch.empty_like(vin)
    monkeypatch.setenv("EW_TB2D_VARIANT", form)
    monkeypatch.setenv("EW_TEST_RB2D_STALL", "1")
    ew.ew_filter_apply(g, p, vin, out)  # returns before the kernels run
    with pytest.raises(ew.EWError) as e:
        ew.ew_rayleigh(g, out, nvec=1)
    assert e.value.status == 6  # EW_ETIMEOUT
    monkeypatch.delenv("EW_TEST_RB2D_STALL")
    ew.ew_filter_apply(g, p, vin, out)
    monkeypatch.setenv("EW_TB2D_VARIANT", "0")
    ref = torch.empty_like(vin)
    ew.ew_filter_apply(g, p, vin, ref)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    ew.ew_rayleigh(g, out, nvec=1)  # no stale report left behind
    g.close()


@pytest.mark.parametrize("n,order", [((2047, 3071), 4), ((5, 3), 4), ((3, 200), 2), ((129, 7), 4), ((301, 97), 2),
                                     ((116, 84), 4), ((117, 85), 4)])
def test_tma_staged_forms_bit_identical(ew, n, order, monkeypatch):
    """Every TMA-staged variant against the shared-memory form (variant 0), bit
    for bit: the full-size rectangle, boxes narrower than the halo (the
    reflection wraps across the whole axis), one-tile and ragged grids, two
    vectors (one tensor-map plane each)."""
    L = tuple(0.01 * x for x in n)
    omega = 120.0 if n[0] > 1000 else 30.0
    monkeypatch.setenv("EW_TB2D_VARIANT", "0")
    _, ref, _ = _run(ew, n, L, order, "fp32", omega, nvec=2, seed=31)
    count = 0
    for i in range(16):
        monkeypatch.setenv("EW_TB2D_VARIANT", "tma:%d" % i)
        try:
            _, out, _ = _run(ew, n, L, order, "fp32", omega, nvec=2, seed=31)
        except ew.EWError as e:
            assert "EW_TB2D_VARIANT" in str(e)
            break
        assert np.array_equal(out, ref), "TMA variant %d differs" % i
        count += 1
    assert count >= 4


@pytest.mark.parametrize("k", [(2, 3, 4), (19, 17, 21)])
def test_cube_511_mode_amplification(ew, k):
    """Full-size 3D workload (511^3, order 2, FP32, CFL 0.8, omega = 60, one
    period) through the launch configuration the bench times (temporally
    blocked 2.5D kernel at its tuned depth): a sine mode is an eigenvector of S,
    so S phi_k = beta~_d(lambda_k) phi_k (eq. correctedBeta with the time
    correction of eq. discreteExplicitLambdaTilde).  A low mode and one near
    the peak; FP32 error bound 4 N_t eps relative."""
    n, L, omega = (511, 511, 511), (1.0, 1.0, 1.0), 60.0
    og = O.Grid(n, L, 2)
    phi = O.sine_mode(og, k)
    lam = math.sqrt(O.lambda2_closed_form(og, [k])[0])
    g = ew.ew_grid_create(3, n, L, order=2, prec="fp32")
    p = ew.filter_params(omega)
    info, _ = ew.ew_filter_setup(g, p)
    vin = torch.tensor(phi, dtype=torch.float32, device="cuda")
    vout = torch.empty_like(vin)
    ew.ew_filter_apply(g, p, vin, vout)
    torch.cuda.synchronize()
    beta = O.beta_tilde(lam, O.filter_params(omega, 1, info["steps_per_period"]))[0]
    err = np.linalg.norm(vout.cpu().double().numpy() - beta * phi) / np.linalg.norm(phi)
    assert err < 4 * info["Nt"] * EPS32, (err, beta)
    g.close()
