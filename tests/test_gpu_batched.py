"""Batched wave-solves of uneven problems (one graph-captured launch
sequence) against the oracle and against the single-problem path.

Tolerances: FP64 to 1e-12 relative (as the single path); the batched tile
step does the same operations per point as the single-grid blocked kernel,
so FP32 results on grids above the one-CTA size agree bit for bit."""
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


def _batch(ew, probs, prec, order):
    dt = torch.float32 if prec == "fp32" else torch.float64
    grids, params, vin, vout, vs = [], [], [], [], []
    for q, (n, L, w) in enumerate(probs):
        g = ew.ew_grid_create(2, n, L, order=order, prec=prec)
        v = ew_inputs.uniform_pm1(100 + q, g.size)
        grids.append(g)
        params.append(ew.filter_params(w))
        vs.append(v)
        vin.append(torch.tensor(v, dtype=dt, device="cuda"))
        vout.append(torch.full_like(vin[-1], float("nan")))
    ew.ew_filter_apply_batched(grids, params, vin, vout)
    torch.cuda.synchronize()
    return grids, params, vin, vout, vs


PROBS = [((300, 70), (1.0, 0.7), 23.0), ((129, 33), (1.3, 0.5), 40.0), ((64, 200), (0.6, 1.9), 12.5),
         ((1, 7), (0.3, 0.9), 9.0), ((255, 255), (1.0, 1.0), 55.0), ((511, 127), (2.0, 0.5), 31.0)]


@pytest.mark.parametrize("order", [2, 4])
def test_batched_fp64_matches_oracle(ew, order):
    grids, params, vin, vout, vs = _batch(ew, PROBS, "fp64", order)
    for q, (n, L, w) in enumerate(PROBS):
        info, _ = ew.ew_filter_setup(grids[q], params[q])
        ref = O.filter_explicit(O.Grid(n, L, order), O.filter_params(w, 1, info["steps_per_period"]), vs[q])
        err = np.max(np.abs(vout[q].cpu().numpy() - ref)) / np.max(np.abs(ref))
        assert err < 1e-12, (q, err)
    for g in grids:
        g.close()


def test_batched_fp32_bitwise_equals_single(ew):
    probs = [p for p in PROBS if p[0][0] * p[0][1] > 16384]
    grids, params, vin, vout, _ = _batch(ew, probs, "fp32", 4)
    for q in range(len(probs)):
        out = torch.empty_like(vin[q])
        ew.ew_filter_apply(grids[q], params[q], vin[q], out)
        torch.cuda.synchronize()
        assert torch.equal(out, vout[q]), q
    for g in grids:
        g.close()


def test_batched_uneven_boxes_workload(ew):
    """The 64-box workload: side lengths in [0.5, 2], n x n grids with n
    log-uniform in [255, 2047], omega in [10, 200], order 2, FP32, all in one
    batched call.  Three problems are compared with the single-problem path
    bit for bit and one with the closed-form single-mode amplification."""
    boxes = ew_inputs.batched_boxes(ew_inputs.BASE_SEED + 3)
    assert len(boxes) == 64
    probs = [(b["n"], b["length"], b["omega"]) for b in boxes]
    grids, params, vin, vout, _ = _batch(ew, probs, "fp32", 2)
    for q in (0, 17, 63):
        out = torch.empty_like(vin[q])
        ew.ew_filter_apply(grids[q], params[q], vin[q], out)
        torch.cuda.synchronize()
        assert torch.equal(out, vout[q]), q
    for g in grids:
        g.close()
    # single mode through the batch, on the smallest box
    q = int(np.argmin([b["n"][0] for b in boxes]))
    n, L, w = probs[q]
    og = O.Grid(n, L, 2)
    k = (3, 4)
    phi = O.sine_mode(og, k)
    g = ew.ew_grid_create(2, n, L, order=2, prec="fp32")
    p = ew.filter_params(w)
    info, _ = ew.ew_filter_setup(g, p)
    x = torch.tensor(phi, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    ew.ew_filter_apply_batched([g, g], [p, p], [x, x], [y, torch.empty_like(x)])
    torch.cuda.synchronize()
    beta = O.beta_tilde(math.sqrt(O.lambda2_closed_form(og, [k])[0]),
                        O.filter_params(w, 1, info["steps_per_period"]))[0]
    err = np.linalg.norm(y.cpu().double().numpy() - beta * phi) / np.linalg.norm(phi)
    assert err < 4 * info["Nt"] * np.finfo(np.float32).eps
    g.close()


def test_batched_fp32_large_box_runs_alone_same_bits(ew):
    """In FP32 a problem whose points x vectors fill the GPU three times over
    with 116 x 88 tiles runs alone inside the batched call (the tuned
    single-problem kernel) while the others share the batched launch; every
    problem's result equals its own ew_filter_apply call bit for bit."""
    props = torch.cuda.get_device_properties(0)
    big = 3 * props.multi_processor_count * 116 * 88
    probs = [((2047, 1535), (1.0, 0.75), 20.0, 2), ((300, 170), (1.0, 0.6), 35.0, 1),
             ((511, 383), (1.2, 0.9), 50.0, 3)]
    assert probs[0][0][0] * probs[0][0][1] * probs[0][3] >= big
    assert all(n[0] * n[1] * k < big for n, _, _, k in probs[1:])
    grids, params, vin, vout = [], [], [], []
    for q, (n, L, w, k) in enumerate(probs):
        g = ew.ew_grid_create(2, n, L, order=4, prec="fp32")
        grids.append(g)
        params.append(ew.filter_params(w))
        vin.append(torch.tensor(ew_inputs.uniform_pm1(200 + q, g.size * k), dtype=torch.float32, device="cuda"))
        vout.append(torch.full_like(vin[-1], float("nan")))
    ew.ew_filter_apply_batched(grids, params, vin, vout, nvec=[k for *_, k in probs])
    torch.cuda.synchronize()
    for q, (_, _, _, k) in enumerate(probs):
        out = torch.empty_like(vin[q])
        ew.ew_filter_apply(grids[q], params[q], vin[q], out, nvec=k)
        torch.cuda.synchronize()
        assert torch.equal(out, vout[q]), q
    for g in grids:
        g.close()
