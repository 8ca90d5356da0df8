"""Host-side checks of the C ABI (no GPU): every declared symbol is exported,
the parameter math (a1) equals the oracle's, and bad arguments are refused."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ew():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_2507_18282_gb300 as ew
    return ew


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ew_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(ew):
    names = _declared_functions()
    assert "ew_filter_apply" in names and "ew_grid_create" in names
    lib = ctypes.CDLL(ew.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("dim,n,length,order,omega,spp,Np,adjust", [
    (2, (63, 63), (1.0, 1.0), 2, 20.0, 0, 1, False),
    (2, (2047, 3071), (1.0, 1.5), 4, 150.0, 0, 2, False),
    (3, (511, 511, 511), (1.0, 1.0, 1.0), 2, 60.0, 0, 1, False),
    (3, (255, 255, 255), (1.0, 1.0, 1.0), 4, 80.0, 10, 3, True),
])
def test_filter_parameters_match_oracle(ew, dim, n, length, order, omega, spp, Np, adjust):
    from oracle import oracle as O
    g = ew.ew_grid_create(dim, n, length, order=order, prec="fp32")
    scheme = "implicit" if adjust else "explicit"
    p = ew.filter_params(omega, num_periods=Np, steps_per_period=spp, scheme=scheme, adjust_omega=adjust)
    info, c = ew.ew_filter_setup(g, p)
    og = O.Grid(n, length, order)
    s = spp if spp else O.steps_per_period_cfl(og, omega, 0.8)
    ref = O.filter_params(omega, Np, s, adjust=adjust)
    assert info["steps_per_period"] == s and info["Nt"] == ref["Nt"]
    assert abs(info["dt"] - ref["dt"]) <= 1e-15 * ref["dt"]
    assert abs(info["omega"] - ref["omega"]) <= 1e-14 * ref["omega"]
    assert abs(info["alpha_d"] - ref["alpha_d"]) <= 1e-14
    np.testing.assert_allclose(c, ref["c"], rtol=0, atol=1e-15 * np.max(np.abs(ref["c"])))
    g.close()


def test_config_steps_per_period(ew):
    """Steps per period at CFL 0.8 of the explicit workloads."""
    cases = [((63, 63), (1.0, 1.0), 2, 20.0, 36), ((2047, 3071), (1.0, 1.5), 4, 150.0, 176),
             ((511, 511, 511), (1.0, 1.0, 1.0), 2, 60.0, 117)]
    for n, L, o, w, want in cases:
        g = ew.ew_grid_create(len(n), n, L, order=o)
        info, _ = ew.ew_filter_setup(g, ew.filter_params(w))
        assert info["steps_per_period"] == want
        g.close()


def test_bad_arguments_are_refused(ew):
    with pytest.raises(ew.EWError) as e:
        ew.ew_grid_create(4, (3, 3, 3), (1, 1, 1))
    assert e.value.status == 1
    with pytest.raises(ew.EWError):
        ew.ew_grid_create(2, (0, 3), (1, 1))
    with pytest.raises(ew.EWError):
        ew.ew_grid_create(2, (3, 3), (1, -1))
    with pytest.raises(ew.EWError):
        ew.ew_grid_create(2, (3, 3), (1, 1), order=3)
    for n in [(1 << 30, 1 << 30, 1 << 30), (1 << 20, 1 << 20, 2)]:  # N would overflow / pass 2^40
        with pytest.raises(ew.EWError) as e:
            ew.ew_grid_create(3, n, (1, 1, 1))
        assert e.value.status == 1 and "2^40" in ew.ew_last_error()
    ew.ew_grid_create(3, (1 << 13, 1 << 13, 1 << 13), (1, 1, 1)).close()  # creation allocates nothing
    g = ew.ew_grid_create(2, (31, 31), (1, 1))
    for p in [ew.filter_params(-1.0), ew.filter_params(5.0, num_periods=0),
              ew.filter_params(5.0, steps_per_period=3),  # beyond the leapfrog stability limit
              ew.filter_params(5.0, steps_per_period=4, scheme="implicit", adjust_omega=True)]:
        with pytest.raises(ew.EWError) as e:
            ew.ew_filter_setup(g, p)
        assert e.value.status == 1
        assert ew.ew_last_error()
    g.close()


def test_wave_solve_length_is_bounded(ew):
    """N_t stays below 2^31 - 1: a tiny omega on a fine grid (CFL-derived steps
    per period beyond int range) and N_p x N_its past the limit are refused with
    EW_EINVAL instead of overflowing or allocating a weight table of that size."""
    g = ew.ew_grid_create(2, (2047, 3071), (1.0, 1.5), order=4)
    with pytest.raises(ew.EWError) as e:
        ew.ew_filter_setup(g, ew.filter_params(1e-9))
    assert e.value.status == 1 and "omega too small" in ew.ew_last_error()
    with pytest.raises(ew.EWError) as e:
        ew.ew_filter_setup(g, ew.filter_params(150.0, num_periods=(1 << 31) // 176 + 1))
    assert e.value.status == 1 and "2^31" in ew.ew_last_error()
    info, _ = ew.ew_filter_setup(g, ew.filter_params(150.0, num_periods=1024))
    assert info["Nt"] == 1024 * 176
    g.close()


def test_every_entry_point_converts_host_exceptions(ew):
    """No C++ exception crosses the ABI: every exported function that returns
    an ew_status is a function-try-block whose handler maps the exception to a
    status (abi_exception)."""
    src = ""
    csrc = os.path.join(ROOT, "paper_2507_18282_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith(".cu"):
            src += open(os.path.join(csrc, f)).read()
    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ew.h")).read(), flags=re.S)
    entry = re.findall(r"\bew_status\s+(ew_[a-z0-9_]+)\s*\(", hdr)
    assert len(entry) >= 15
    for name in entry:
        m = re.search(r"ew_status\s+" + name + r"\s*\([^;{]*?\)\s*(try)?\s*\{", src, flags=re.S)
        assert m, name
        assert m.group(1) == "try", name


def test_neumann_faces_add_active_wall_points(ew):
    """A Neumann face's wall points are active: one more point per Neumann
    face along its axis; h stays length / (n + 1), so the explicit step limit
    (the largest eigenvalue is the same 4 sum 1/h^2, resp. 16/3 sum 1/h^2) and
    the parameters of a wave-solve do not change."""
    g = ew.ew_grid_create(3, (10, 12, 7), (1.0, 1.2, 0.7), order=4, bc=("N", "D", "N", "N", "D", "N"))
    assert g.n == (11, 14, 8) and g.size == 11 * 14 * 8
    gd = ew.ew_grid_create(3, (10, 12, 7), (1.0, 1.2, 0.7), order=4)
    p = ew.filter_params(7.0, num_periods=3)
    a, wa = ew.ew_filter_setup(g, p)
    b, wb = ew.ew_filter_setup(gd, p)
    assert a == b and np.array_equal(wa, wb)
    g.close()
    gd.close()
    with pytest.raises(ValueError):
        ew.ew_grid_create(2, (3, 3), (1, 1), bc=("N", "D"))
    with pytest.raises(ew.EWError) as e:
        ew.ew_grid_create(2, (3, 3), (1, 1), bc=(0, 1, 2, 0))   # 2 is not a boundary kind
    assert e.value.status == 1


def test_mapped_grid_creation_and_step_limit(ew):
    """Creating a curvilinear grid needs no GPU; a map that folds over (J <= 0)
    is refused; the explicit step limit comes from a Gershgorin bound of
    rho(-L), which must not be below the true spectral radius (the oracle's
    dense operator)."""
    import ew_inputs
    from oracle import oracle as O
    n = (14, 11)
    xy = ew_inputs.mapped_vertices(*n, "square_warp", eps=0.15)
    g = ew.ew_grid_create_mapped(n, xy, prec="fp64")
    assert g.size == n[0] * n[1]
    info, _ = ew.ew_filter_setup(g, ew.filter_params(9.0, steps_per_period=0))
    g.close()
    L = np.stack([O.mapped_apply_L(O.MappedGrid(n, xy), e) for e in np.eye(n[0] * n[1])], axis=1)
    rho = np.max(np.abs(np.linalg.eigvals(L)))
    # leapfrog is stable for dt^2 rho / 4 <= 1; the library's dt must satisfy it
    assert info["dt"] ** 2 * rho / 4.0 <= 1.0
    bad = xy.copy()
    bad[..., 0] = -bad[..., 0]  # mirror: orientation reversed, J < 0
    with pytest.raises(ew.EWError) as e:
        ew.ew_grid_create_mapped(n, bad)
    assert e.value.status == 1


def test_pair_precision_is_two_dimensional(ew):
    g = ew.ew_grid_create(2, (20, 30), (1.0, 1.5), order=4, prec="fp32x2")
    assert g.size == 600
    g.close()
    with pytest.raises(ew.EWError) as e:
        ew.ew_grid_create(3, (8, 8, 8), (1.0, 1.0, 1.0), prec="fp32x2")
    assert e.value.status == 7


def test_binding_checks_buffers_before_the_call(ew):
    """The binding refuses what the library cannot check itself: host tensors
    for device pointers, and a per-problem vector count list of the wrong length."""
    import torch
    with pytest.raises(TypeError):
        ew.mg_params(learned_levels=1, weights=torch.zeros(432, dtype=torch.float32))
    g = ew.ew_grid_create(2, (15, 15), (1.0, 1.0))
    with pytest.raises(ValueError):
        ew.ew_filter_apply_batched([g, g], [ew.filter_params(5.0)] * 2, [None, None], [None, None], nvec=[1])
    with pytest.raises(TypeError):
        x = torch.zeros(g.size, dtype=torch.float32)
        ew.ew_filter_apply(g, ew.filter_params(5.0), x, torch.zeros_like(x))
    g.close()


def test_every_entry_point_refuses_null_arguments(ew):
    """Each exported function, called with null pointers and zero sizes, returns
    an error status and a message instead of dereferencing them (run in a
    child process, so that a crash would fail this test rather than the run)."""
    script = r'''
import ctypes
from paper_2507_18282_gb300 import _lib as L
lib = L.lib
calls = {
    "ew_grid_create": (2, None, None, 2, None, 0, None),
    "ew_grid_create_mapped": (None, None, 0, None),
    "ew_filter_setup": (None, None, None, None, 0),
    "ew_filter_apply": (None, None, None, None, 1, None),
    "ew_filter_apply_host": (None, None, None, None, 1, 0, None),
    "ew_filter_apply_batched": (0, None, None, None, None, None, None),
    "ew_filter_apply_noalloc": (None, None, None, None, None),
    "ew_choose_num_periods": (None, None, 1, 2, 1, None, None),
    "ew_apply_L": (None, None, None, 1, None),
    "ew_rayleigh": (None, None, 1, None, None, None),
    "ew_power_iteration": (None, None, None, 1, 0.0, None, None, None, None),
    "ew_arnoldi_eigs": (None, None, None, None, None, None, None, None),
    "ew_arnoldi_eigs_batched": (0, None, None, None, None, None, None, None, None, None),
    "ew_tuned_variant": (None, 1, None, 0, None, None, None),
    "ew_implicit_step_mg": (None, 0.0, None, None, None, None, None, None),
    "ew_smoother_forward": (None, None, None, None, None),
    "ew_smoother_backward": (None, None, None, None, None, None),
    "ew_smoother_train": (None, 0.0, None, None, None, None),
    "ew_profile_read": (None,),
}
for name, args in calls.items():
    st = getattr(lib, name)(*args)
    assert st in (L.EW_EINVAL, L.EW_ECUDA), (name, st)
    assert lib.ew_last_error(), name
lib.ew_grid_destroy(None)
print("ok", len(calls))
'''
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", script], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == "ok 19"


def test_header_is_plain_c(ew, tmp_path):
    """include/ew.h compiles as C99 (the ABI is a C interface, usable without
    C++) and a C program links against the library's exported names."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    inc = next((os.path.join(d, "include") for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda")
                if d and os.path.exists(os.path.join(d, "include", "cuda_runtime_api.h"))), None)
    if not cc or not inc:
        pytest.skip("needs gcc and the CUDA headers")
    src = tmp_path / "use_ew.c"
    src.write_text(
        '#include "ew.h"\n'
        "int main(void) {\n"
        "    ew_grid* g = 0;\n"
        "    int64_t n[3] = {15, 15, 1};\n"
        "    double len[3] = {1.0, 1.0, 1.0};\n"
        "    ew_status s = ew_grid_create(2, n, len, 2, 0, EW_FP32, &g);\n"
        "    ew_filter_params p = {0};\n"
        "    ew_filter_info info;\n"
        "    p.omega = 5.0; p.num_periods = 1;\n"
        "    if (s == EW_OK) s = ew_filter_setup(g, &p, &info, 0, 0);\n"
        "    ew_grid_destroy(g);\n"
        "    return (s == EW_OK && info.num_steps > 0) ? 0 : 1;\n"
        "}\n")
    exe = tmp_path / "use_ew"
    libdir = os.path.dirname(ew.LIB_PATH)
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I", inc,
                           str(src), "-L", libdir, "-lew", "-Wl,-rpath," + libdir, "-o", str(exe)])
    assert subprocess.run([str(exe)], timeout=120).returncode == 0
