"""GPU multigrid, implicit wave-solve and learned smoother (row a6) against
the oracle.

Tolerances: FP64 V-cycles and implicit wave-solves repeat the oracle's cycle
operation for operation (only rounding order differs), so 1e-12 relative.
The learned smoother rounds its input and hidden activations to BF16
(8 significant bits: at most 2^-8 relative per rounding), so forward outputs
agree with the FP64 oracle to about 2^-8 in the 2-norm (4e-3 used); gradients
to 1e-2.  Element-wise bounds at larger sizes: test_gpu_learned.py.
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


def _config5_a(h=1.0 / 256):
    """a = dt^2 / 2 of the 255^3 implicit workload: omega = 80 adjusted to
    omega~ for 10 steps per period (eq. adjustedOmega), dt = 2 pi / (10 omega~)."""
    prm = O.filter_params(80.0, 1, 10, adjust=True)
    return 0.5 * prm["dt"] ** 2


@pytest.mark.parametrize("n,order", [((31, 31, 31), 4), ((63, 63), 2), ((15, 31, 7), 2)])
def test_vcycle_parity_fp64(ew, n, order):
    L = tuple(1.0 for _ in n)
    g = ew.ew_grid_create(len(n), n, L, order=order, prec="fp64")
    og = O.Grid(n, L, order)
    a = 0.5 * (2 * math.pi / (30.0 * 10)) ** 2
    b = ew_inputs.uniform_pm1(21, og.size)
    x0 = ew_inputs.uniform_pm1(22, og.size)
    x = torch.tensor(x0, device="cuda")
    mg = ew.mg_params(pre=2, post=2, max_cycles=3)
    conv, cyc = ew.ew_implicit_step_mg(g, a, torch.tensor(b, device="cuda"), x, mg)
    ref, hist = O.mg_solve(og, a, b, x0=x0, ncycles=3)
    assert cyc == 3
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    assert abs(conv - (hist[-1] / hist[0]) ** (1 / 3)) < 1e-6
    g.close()


@pytest.mark.parametrize("n,order", [((63, 63), 2), ((15, 31, 7), 2), ((63, 63), 4), ((31, 15, 31), 4)])
def test_red_black_vcycle_parity_fp64(ew, n, order):
    """Multi-colour Gauss-Seidel smoothing (red-black at second order, three
    colours at fourth order): the GPU's colour sweeps against the oracle's
    point-by-point sweeps, three V(2,2) cycles, FP64."""
    L = tuple(1.0 for _ in n)
    g = ew.ew_grid_create(len(n), n, L, order=order, prec="fp64")
    og = O.Grid(n, L, order)
    a = 0.5 * (2 * math.pi / (12.0 * 10)) ** 2
    b = ew_inputs.uniform_pm1(24, og.size)
    x0 = ew_inputs.uniform_pm1(25, og.size)
    x = torch.tensor(x0, device="cuda")
    mg = ew.mg_params(pre=2, post=2, max_cycles=3, red_black=True)
    conv, cyc = ew.ew_implicit_step_mg(g, a, torch.tensor(b, device="cuda"), x, mg)
    ref, hist = O.mg_solve(og, a, b, x0=x0, ncycles=3, red_black=True)
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    jac, _ = ew.ew_implicit_step_mg(g, a, torch.tensor(b, device="cuda"), torch.tensor(x0, device="cuda"),
                                    ew.mg_params(pre=2, post=2, max_cycles=3))
    assert conv < 0.6 * jac
    g.close()


def test_mg_fp32_converges_to_exact_solve(ew):
    n, L = (63, 63, 63), (1.0, 1.0, 1.0)
    g = ew.ew_grid_create(3, n, L, order=4, prec="fp32")
    og = O.Grid(n, L, 4)
    a = _config5_a(1.0 / 64)
    b = ew_inputs.uniform_pm1(23, og.size)
    x = torch.zeros(og.size, dtype=torch.float32, device="cuda")
    mg = ew.mg_params(pre=2, post=2, max_cycles=30, rtol=1e-6)
    conv, cyc = ew.ew_implicit_step_mg(g, a, torch.tensor(b, dtype=torch.float32, device="cuda"), x, mg)
    exact = O.implicit_solve_closed_form(og, a, b)
    assert np.max(np.abs(x.cpu().double().numpy() - exact)) < 1e-5 * np.max(np.abs(exact))
    assert conv < 0.3 and cyc < 30
    g.close()


def test_mg_refuses_grids_that_do_not_coarsen(ew):
    g = ew.ew_grid_create(3, (64, 64, 64), (1, 1, 1), order=2, prec="fp32")
    x = torch.zeros(64 ** 3, device="cuda")
    with pytest.raises(ew.EWError) as e:
        ew.ew_implicit_step_mg(g, 1e-4, x, x.clone(), ew.mg_params())
    assert e.value.status == 7
    g.close()


@pytest.mark.parametrize("n,order,guess", [((31, 31, 31), 4, "rhs"), ((63, 31), 2, "rhs"),
                                           ((31, 15, 31), 4, "previous"), ((63, 31), 2, "previous")])
def test_implicit_wave_solve_parity_fp64(ew, n, order, guess):
    """Implicit wave-solve (adjusted omega, 10 steps per period, 2 V-cycles per
    system) equals the oracle's implicit scheme with its own multigrid, for
    either initial guess of the systems."""
    L = tuple(1.0 for _ in n)
    g = ew.ew_grid_create(len(n), n, L, order=order, prec="fp64")
    og = O.Grid(n, L, order)
    mg = ew.mg_params(pre=2, post=2, max_cycles=2, guess=guess)
    p = ew.filter_params(12.0, num_periods=2, steps_per_period=10, scheme="implicit", adjust_omega=True, mg=mg)
    v = ew_inputs.uniform_pm1(24, og.size)
    vin = torch.tensor(v, device="cuda")
    vout = torch.empty_like(vin)
    ew.ew_filter_apply(g, p, vin, vout)
    torch.cuda.synchronize()
    prm = O.filter_params(12.0, 2, 10, adjust=True)
    ref = O.filter_implicit_mg(og, prm, v, ncycles=2, guess=guess)
    np.testing.assert_allclose(vout.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    g.close()


def test_implicit_mode_amplification_cube_255_order4(ew):
    """Full-size implicit workload (255^3, order 4, FP32, 10 steps per period,
    adjusted omega = 80, 4 V-cycles per system): S phi_k = beta~_d phi_k for the
    implicit time correction (eq. discreteCorr) within the multigrid and FP32
    error (the V-cycle reduces the residual ~10x per cycle)."""
    n, L = (255, 255, 255), (1.0, 1.0, 1.0)
    og = O.Grid(n, L, 4)
    k = (14, 15, 16)
    phi = O.sine_mode(og, k)
    lam = math.sqrt(O.lambda2_closed_form(og, [k])[0])
    g = ew.ew_grid_create(3, n, L, order=4, prec="fp32")
    mg = ew.mg_params(pre=2, post=2, max_cycles=4)
    p = ew.filter_params(80.0, num_periods=1, steps_per_period=10, scheme="implicit", adjust_omega=True, mg=mg)
    vin = torch.tensor(phi, dtype=torch.float32, device="cuda")
    vout = torch.empty_like(vin)
    ew.ew_filter_apply(g, p, vin, vout)
    torch.cuda.synchronize()
    prm = O.filter_params(80.0, 1, 10, adjust=True)
    beta = O.beta_tilde(lam, prm, "implicit")[0]
    err = np.linalg.norm(vout.cpu().double().numpy() - beta * phi) / np.linalg.norm(phi)
    assert err < 1e-3, (err, beta)
    g.close()


def _bf16(x):
    """Round float64 values to the nearest BF16 (ties to even), via float32 bits."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_smoother_forward_parity(ew):
    n = (17, 13, 11)
    og = O.Grid(n, (1.0, 1.0, 1.0), 4)
    g = ew.ew_grid_create(3, n, (1.0, 1.0, 1.0), order=4, prec="fp32")
    w = _bf16(ew_inputs.learned_init(31, 0.3))
    r = _bf16(ew_inputs.uniform_pm1(32, og.size))
    y = torch.empty(og.size, dtype=torch.float32, device="cuda")
    ew.ew_smoother_forward(g, torch.tensor(w, dtype=torch.float32, device="cuda"),
                           torch.tensor(r, dtype=torch.float32, device="cuda"), y)
    torch.cuda.synchronize()
    _, ref = O.conv_net_forward(n, w, r)
    rel = np.linalg.norm(y.cpu().double().numpy() - ref) / np.linalg.norm(ref)
    assert rel < 4e-3, rel
    g.close()


def test_smoother_backward_parity(ew):
    n = (17, 13, 11)
    og = O.Grid(n, (1.0, 1.0, 1.0), 4)
    g = ew.ew_grid_create(3, n, (1.0, 1.0, 1.0), order=4, prec="fp32")
    w = _bf16(ew_inputs.learned_init(33, 0.3))
    r = _bf16(ew_inputs.uniform_pm1(34, og.size))
    gy = ew_inputs.uniform_pm1(35, og.size).astype(np.float32).astype(np.float64)
    grad = torch.empty(432, dtype=torch.float32, device="cuda")
    ew.ew_smoother_backward(g, torch.tensor(w, dtype=torch.float32, device="cuda"),
                            torch.tensor(r, dtype=torch.float32, device="cuda"),
                            torch.tensor(gy, dtype=torch.float32, device="cuda"), grad)
    torch.cuda.synchronize()
    hid, _ = O.conv_net_forward(n, w, r)
    ref, _ = O.conv_net_backward(n, w, r, hid, gy)
    rel = np.linalg.norm(grad.cpu().double().numpy() - ref) / np.linalg.norm(ref)
    assert rel < 1e-2, rel
    g.close()


def test_learned_smoother_beats_plain_multigrid(ew):
    """The learned smoother, trained on the GPU on residuals from plain-MG
    solves of the 255^3 order-4 implicit system, lowers the V(2,2) convergence
    factor below plain damped-Jacobi multigrid on the same system (the acceptance test
    built into the trainer); otherwise the trainer keeps plain multigrid."""
    n = (255, 255, 255)
    g = ew.ew_grid_create(3, n, (1.0, 1.0, 1.0), order=4, prec="fp32")
    a = _config5_a()
    w0 = ew_inputs.learned_init(36, 0.05)
    w = torch.tensor(w0, dtype=torch.float32, device="cuda")
    rep = ew.ew_smoother_train(g, a, w, steps=600, samples=12, lr=5e-3, seed=5)
    assert rep["loss_last"] < rep["loss_first"]
    assert rep["accepted"], rep
    assert rep["conv_learned"] < rep["conv_plain"], rep
    g.close()


def test_mg_guess_must_be_0_or_1(ew):
    g = ew.ew_grid_create(2, (31, 31), (1.0, 1.0), order=2, prec="fp64")
    p = ew.filter_params(12.0, steps_per_period=10, scheme="implicit", mg=ew.mg_params(guess=2))
    x = torch.zeros(g.size, dtype=torch.float64, device="cuda")
    with pytest.raises(ew.EWError, match="EW_EINVAL"):
        ew.ew_filter_apply(g, p, x, torch.empty_like(x))
    g.close()
