"""Learned multigrid smoother on the GPU against the FP64 oracle (row a6):
the forward and backward kernels at a size spanning several z-chunks and
ragged columns of the tensor-core kernel, the learned V-cycle (the in-place
x += N(r) form of the kernels) and the implicit wave-solve with learned
multigrid (eqs. implicitScheme, impMatrix, implicitStep1).

Tolerances come from BF16 rounding.  BF16 keeps 8 significant bits, so one
rounding to nearest errs by at most u = 2^-8 relative.  The weights and the
residual are BF16 values already (rounded here, on both sides), so in the
forward pass only the hidden activations h are rounded: element by element,
|y_gpu - y| <= u sum_c sum_o |W2[c][o]| |h_c(x + o)| plus FP32 accumulation
(27 x 8 terms at 2^-24, bounded by 1e-5 of the same sum).  The weight
gradient dW2 = sum gy h inherits u sum |gy| |h| per component; dW1 takes no
rounded activation.  Inside a V-cycle every learned correction carries such
an error, which the later sweeps and cycles damp: the iterate after a cycle
stays within u times that cycle's correction (a CPU emulation of the
kernels' rounding gives 4e-4 of it for these cases), and the wave-solve
within u of its result."""
import math

import numpy as np
import pytest
import torch

import ew_inputs
from oracle import oracle as O

pytestmark = pytest.mark.gpu
U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def ew():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_18282_gb300 as ew
    return ew


def _bf16(x):
    """Round to the nearest BF16 (ties to even), via the float32 bits."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _corr_abs(n3, field, kernel):
    """sum_o |kernel[o]| |field(x + o)|, zero outside the box (x fastest)."""
    from scipy import ndimage
    f = np.abs(field).reshape(n3[2], n3[1], n3[0])
    k = np.abs(np.asarray(kernel)).reshape(3, 3, 3)
    return ndimage.correlate(f, k, mode="constant", cval=0.0).reshape(-1)


def _config5_a():
    """a = dt^2/2 of the implicit scheme at omega = 80 adjusted for 10 steps per period."""
    return 0.5 * O.filter_params(80.0, 1, 10, adjust=True)["dt"] ** 2


def _jacobi_like(h, a, seed, pert, wJ=0.8, d0=2.5):
    """Seeded smoother weights near the damped-Jacobi correction wJ r / D
    (W1[0] and W2[0] centre taps), every tap and channel perturbed by `pert`
    of its scale, BF16-rounded: a convergent smoother that uses all weights."""
    D = 1.0 + a * sum(d0 / x ** 2 for x in h)
    w = np.zeros(432)
    w[13] = 1.0
    w[216 + 13] = wJ / D
    rnd = ew_inputs.learned_init(seed, 1.0)
    w[:216] += pert * rnd[:216]
    w[216:] += pert * (wJ / D) * rnd[216:]
    return _bf16(w)


FWD_SIZES = [(37, 29, 70), (16, 16, 33)]   # 3 z-chunks with ragged 16 x 16 columns; exact columns, 2 chunks


@pytest.mark.parametrize("n", FWD_SIZES)
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_smoother_forward_elementwise(ew, n, prec):
    og = O.Grid(n, (1.0, 1.0, 1.0), 4)
    g = ew.ew_grid_create(3, n, (1.0, 1.0, 1.0), order=4, prec=prec)
    dt = torch.float32 if prec == "fp32" else torch.float64
    w = _bf16(ew_inputs.learned_init(61, 0.3))
    r = _bf16(ew_inputs.uniform_pm1(62, og.size))
    y = torch.empty(og.size, dtype=dt, device="cuda")
    ew.ew_smoother_forward(g, torch.tensor(w, dtype=torch.float32, device="cuda"),
                           torch.tensor(r, dtype=dt, device="cuda"), y)
    torch.cuda.synchronize()
    hid, ref = O.conv_net_forward(n, w, r)
    W2 = w[216:].reshape(8, 27)
    W1 = w[:216].reshape(8, 27)
    N = og.size
    bound = np.zeros(N)
    for c in range(8):
        bound += (U_BF16 + 1e-5) * _corr_abs(n, hid[c * N:(c + 1) * N], W2[c])
        bound += 1e-5 * _corr_abs(n, _corr_abs(n, r, W1[c]), W2[c])
    diff = np.abs(y.cpu().double().numpy() - ref)
    assert np.all(diff <= bound), (np.max(diff / np.maximum(bound, 1e-300)), np.argmax(diff - bound))
    g.close()


@pytest.mark.parametrize("n", FWD_SIZES)
def test_smoother_backward_elementwise(ew, n):
    og = O.Grid(n, (1.0, 1.0, 1.0), 4)
    g = ew.ew_grid_create(3, n, (1.0, 1.0, 1.0), order=4, prec="fp32")
    w = _bf16(ew_inputs.learned_init(63, 0.3))
    r = _bf16(ew_inputs.uniform_pm1(64, og.size))
    gy = ew_inputs.uniform_pm1(65, og.size).astype(np.float32).astype(np.float64)
    grad = torch.empty(432, dtype=torch.float32, device="cuda")
    ew.ew_smoother_backward(g, torch.tensor(w, dtype=torch.float32, device="cuda"),
                            torch.tensor(r, dtype=torch.float32, device="cuda"),
                            torch.tensor(gy, dtype=torch.float32, device="cuda"), grad)
    torch.cuda.synchronize()
    hid, _ = O.conv_net_forward(n, w, r)
    ref, _ = O.conv_net_backward(n, w, r, hid, gy)
    got = grad.cpu().double().numpy()
    N = og.size
    # dW2[c][o] = sum_x gy(x) h_c(x + o): the rounded h gives at most u sum |gy| |h_c(x + o)|
    bound = np.zeros(432)
    ag = np.abs(gy).reshape(n[2], n[1], n[0])
    for c in range(8):
        ah = np.abs(hid[c * N:(c + 1) * N]).reshape(n[2], n[1], n[0])
        hp = np.pad(ah, 1)
        t = 0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    sh = hp[1 + dz:1 + dz + n[2], 1 + dy:1 + dy + n[1], 1 + dx:1 + dx + n[0]]
                    bound[216 + c * 27 + t] = U_BF16 * float(np.sum(ag * sh))
                    t += 1
    # FP32 rounding of the result and of the accumulated terms
    bound += 1e-6 * np.max(np.abs(ref)) + 2.0 ** -23 * np.abs(ref)
    diff = np.abs(got - ref)
    assert np.all(diff <= bound), np.max(diff / bound)
    # dW1 takes no rounded activation: FP32-level agreement
    assert np.max(np.abs(got[:216] - ref[:216])) <= 1e-5 * np.max(np.abs(ref[:216]))
    g.close()


MG_N = (39, 31, 71)   # coarsens 39x31x71 -> 19x15x35 -> 9x7x17 -> 4x3x8


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("cycles", [1, 2])
def test_learned_vcycle_parity(ew, prec, levels, cycles):
    """ew_implicit_step_mg with learned_levels = 1, 2 (V(2,2)) against the
    oracle's mg_solve with the same weights."""
    L = (1.0, 1.0, 1.0)
    og = O.Grid(MG_N, L, 4)
    g = ew.ew_grid_create(3, MG_N, L, order=4, prec=prec)
    dt = torch.float32 if prec == "fp32" else torch.float64
    a = _config5_a()
    nets = np.stack([_jacobi_like(og.h, a, 71, 0.03),
                     _jacobi_like(tuple(2 * x for x in og.h), a, 72, 0.03)])[:levels]
    b = ew_inputs.uniform_pm1(73, og.size)
    x0 = ew_inputs.uniform_pm1(74, og.size)
    if prec == "fp32":
        b = b.astype(np.float32).astype(np.float64)
        x0 = x0.astype(np.float32).astype(np.float64)
    wts = torch.tensor(nets.reshape(-1), dtype=torch.float32, device="cuda")
    x = torch.tensor(x0, dtype=dt, device="cuda")
    mg = ew.mg_params(pre=2, post=2, max_cycles=cycles, learned_levels=levels, weights=wts)
    conv, cyc = ew.ew_implicit_step_mg(g, a, torch.tensor(b, dtype=dt, device="cuda"), x, mg)
    ref, hist = O.mg_solve(og, a, b, x0=x0, ncycles=cycles, net=nets)
    prev = x0 if cycles == 1 else O.mg_solve(og, a, b, x0=x0, ncycles=cycles - 1, net=nets)[0]
    got = x.cpu().double().numpy()
    assert cyc == cycles
    assert np.max(np.abs(got - ref)) <= U_BF16 * np.max(np.abs(ref - prev))
    assert abs(conv - (hist[-1] / hist[0]) ** (1.0 / cycles)) <= 0.05 * conv
    g.close()


@pytest.mark.parametrize("cycles", [1, 2])
def test_learned_implicit_wave_solve_parity(ew, cycles):
    """FP32 implicit wave-solve (omega = 80 adjusted, 10 steps per period, one
    period) with learned multigrid on the finest level against the oracle's
    implicit scheme with its own learned multigrid, same weights."""
    L = (1.0, 1.0, 1.0)
    og = O.Grid(MG_N, L, 4)
    g = ew.ew_grid_create(3, MG_N, L, order=4, prec="fp32")
    prm = O.filter_params(80.0, 1, 10, adjust=True)
    a = 0.5 * prm["dt"] ** 2
    net = _jacobi_like(og.h, a, 75, 0.03)
    wts = torch.tensor(net, dtype=torch.float32, device="cuda")
    mg = ew.mg_params(pre=2, post=2, max_cycles=cycles, learned_levels=1, weights=wts)
    p = ew.filter_params(80.0, num_periods=1, steps_per_period=10, scheme="implicit", adjust_omega=True, mg=mg)
    info, _ = ew.ew_filter_setup(g, p)
    assert info["Nt"] == prm["Nt"] and abs(info["dt"] - prm["dt"]) <= 1e-15 * prm["dt"]
    v = ew_inputs.uniform_pm1(76, og.size).astype(np.float32).astype(np.float64)
    vin = torch.tensor(v, dtype=torch.float32, device="cuda")
    vout = torch.empty_like(vin)
    ew.ew_filter_apply(g, p, vin, vout)
    torch.cuda.synchronize()
    ref = O.filter_implicit_mg(og, prm, v, ncycles=cycles, net=net[None, :])
    got = vout.cpu().double().numpy()
    assert np.max(np.abs(got - ref)) <= U_BF16 * np.max(np.abs(ref))
    g.close()


def test_learned_implicit_mode_amplification_cube_255(ew):
    """Full-size implicit workload (255^3, order 4, FP32, omega = 80 adjusted,
    10 steps per period) with the learned smoother on the finest level (seeded
    near-Jacobi weights, 4 V(2,2) cycles per system): the tensor-core smoother
    over all 8 z-chunks.  S phi_k = beta~_d phi_k (eq. discreteCorr) within the
    multigrid, BF16 and FP32 error."""
    n, L = (255, 255, 255), (1.0, 1.0, 1.0)
    og = O.Grid(n, L, 4)
    k = (14, 15, 16)
    phi = O.sine_mode(og, k)
    lam = math.sqrt(O.lambda2_closed_form(og, [k])[0])
    prm = O.filter_params(80.0, 1, 10, adjust=True)
    a = 0.5 * prm["dt"] ** 2
    g = ew.ew_grid_create(3, n, L, order=4, prec="fp32")
    wts = torch.tensor(_jacobi_like(og.h, a, 77, 0.03), dtype=torch.float32, device="cuda")
    mg = ew.mg_params(pre=2, post=2, max_cycles=4, learned_levels=1, weights=wts)
    p = ew.filter_params(80.0, num_periods=1, steps_per_period=10, scheme="implicit", adjust_omega=True, mg=mg)
    vin = torch.tensor(phi, dtype=torch.float32, device="cuda")
    vout = torch.empty_like(vin)
    ew.ew_filter_apply(g, p, vin, vout)
    torch.cuda.synchronize()
    beta = O.beta_tilde(lam, prm, "implicit")[0]
    err = np.linalg.norm(vout.cpu().double().numpy() - beta * phi) / np.linalg.norm(phi)
    assert err < 1e-3, (err, beta)
    g.close()


@pytest.mark.parametrize("levels", [1, 2])
def test_composed_smoother_vcycle_to_fp32_rounding(ew, levels):
    """Inside the V-cycle on FP32 grids the learned smoother runs as its composed
    5x5x5 stencil (the layers are linear, so W2 after W1 is one stencil; outputs
    on a wall plane use the stencil of their wall class, since hidden points
    beyond the wall are zero).  With the hidden activations no longer rounded to
    BF16, the cycle matches the oracle's two-layer FP64 cycle to FP32 rounding:
    within 1e-5 of the cycle's correction, element by element (39 x 31 x 71 and
    19 x 15 x 35: ragged 128 x 8 x 32 tiles, every wall class)."""
    L = (1.0, 1.0, 1.0)
    og = O.Grid(MG_N, L, 4)
    g = ew.ew_grid_create(3, MG_N, L, order=4, prec="fp32")
    a = _config5_a()
    nets = np.stack([_jacobi_like(og.h, a, 81, 0.03),
                     _jacobi_like(tuple(2 * x for x in og.h), a, 82, 0.03)])[:levels]
    b = ew_inputs.uniform_pm1(83, og.size).astype(np.float32).astype(np.float64)
    x0 = ew_inputs.uniform_pm1(84, og.size).astype(np.float32).astype(np.float64)
    wts = torch.tensor(nets.reshape(-1), dtype=torch.float32, device="cuda")
    x = torch.tensor(x0, dtype=torch.float32, device="cuda")
    mg = ew.mg_params(pre=2, post=2, max_cycles=1, learned_levels=levels, weights=wts)
    ew.ew_implicit_step_mg(g, a, torch.tensor(b, dtype=torch.float32, device="cuda"), x, mg)
    ref, _ = O.mg_solve(og, a, b, x0=x0, ncycles=1, net=nets)
    got = x.cpu().double().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref - x0))
    g.close()
