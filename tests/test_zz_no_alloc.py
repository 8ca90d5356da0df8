"""ew_filter_apply_noalloc: the wave-solve for callers that cannot allocate
device memory (plugins whose host application owns every allocation, real-time
loops that must not enter the allocator).  Its scratch is a fixed device
array inside the library, so it is checked against ew_filter_apply, which
allocates its own, on two calls in a row; before the checked calls another
call on a different, larger grid leaves other contents in the shared array,
so a kernel that read something the call did not write itself would show.

Tolerances as in the filter parity tests: FP64 1e-12 relative in the max
norm; FP32 ||difference||_2 / ||v||_2 <= 4 N_t eps32.  This file is collected
last so that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import ew_inputs

pytestmark = pytest.mark.gpu
EPS32 = float(np.finfo(np.float32).eps)


@pytest.fixture(scope="module")
def ew():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_18282_gb300 as ew
    return ew


def _noalloc(ew, g, p, vin, vout):
    """The C ABI entry point, called directly (argument marshalling only)."""
    st = ew._lib.lib.ew_filter_apply_noalloc(g.handle, ctypes.byref(p), ctypes.c_void_p(vin.data_ptr()),
                                             ctypes.c_void_p(vout.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def _fill_array_with_another_grid(ew, prec):
    """One call on a larger grid of another shape: the shared array then holds
    that grid's time levels where the checked call's padding and tails lie."""
    g = ew.ew_grid_create(2, (700, 511), (1.3, 0.9), order=2, prec=prec)
    p = ew.filter_params(90.0)
    dt = torch.float32 if prec == "fp32" else torch.float64
    vin = torch.tensor(ew_inputs.uniform_pm1(77, g.size), dtype=dt, device="cuda")
    out = torch.empty_like(vin)
    assert _noalloc(ew, g, p, vin, out) == 0, ew.ew_last_error()
    torch.cuda.synchronize()
    g.close()


@pytest.mark.parametrize("dim,n,L,order,prec,omega", [
    (2, (300, 170), (1.0, 0.6), 4, "fp32", 35.0),
    (2, (97, 61), (1.0, 0.7), 2, "fp32", 25.0),     # small: ew_filter_apply takes its one-CTA path
    (3, (45, 40, 33), (1.0, 0.9, 0.8), 2, "fp64", 20.0),
])
def test_noalloc_matches_allocating_path_on_two_calls(ew, dim, n, L, order, prec, omega):
    _fill_array_with_another_grid(ew, prec)
    g = ew.ew_grid_create(dim, n, L, order=order, prec=prec)
    p = ew.filter_params(omega)
    info, _ = ew.ew_filter_setup(g, p)
    dt = torch.float32 if prec == "fp32" else torch.float64
    for call in range(2):
        v = ew_inputs.uniform_pm1(500 + call, g.size)
        vin = torch.tensor(v, dtype=dt, device="cuda")
        ref = torch.empty_like(vin)
        ew.ew_filter_apply(g, p, vin, ref)
        out = torch.full_like(vin, float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = _noalloc(ew, g, p, vin, out)
        torch.cuda.synchronize()
        assert st == 0, ew.ew_last_error()
        if call == 1:  # after a first call (kernels loaded): the device's free memory is unchanged
            assert torch.cuda.mem_get_info()[0] == free_before
        a, b = out.cpu().double().numpy(), ref.cpu().double().numpy()
        assert np.all(np.isfinite(a))
        if prec == "fp64":
            assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))
        else:
            assert np.linalg.norm(a - b) / np.linalg.norm(v) < 4 * info["Nt"] * EPS32
    g.close()


def test_noalloc_rejects_sizes_beyond_its_array(ew):
    g = ew.ew_grid_create(2, (2047, 3071), (1.0, 1.5), order=4, prec="fp32")
    p = ew.filter_params(150.0)
    x = torch.zeros(g.size, dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(ew, g, p, x, y) == 1
    assert "at most" in ew.ew_last_error()
    g.close()


def test_noalloc_rejects_a_negative_temporal_block(ew):
    g = ew.ew_grid_create(2, (100, 80), (1.0, 0.8), order=2, prec="fp32")
    p = ew.filter_params(20.0, temporal_block=-1)
    x = torch.zeros(g.size, dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(ew, g, p, x, y) == 1
    assert "temporal_block" in ew.ew_last_error()
    g.close()
