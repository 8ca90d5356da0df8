"""The boundary closure of the box kernels as an extension map
(paper_2507_18282_gb300/csrc/ew_bc_dev.cuh, compiled for the host; no GPU),
checked against its definition rather than against a second formula.

For an axis with active points 0 .. n-1 the extension E of a grid function u
is fixed by: E = u on the active points; E = 0 on a Dirichlet wall (index -1
below, n above); and reflection about each wall, odd at a Dirichlet wall
(u = 0 and u_xx = 0 there: the order-4 closure) and even at a Neumann wall
(the symmetry plane at index 0 below, n-1 above):
    E(w_lo - d) = s_lo E(w_lo + d),   E(w_hi + d) = s_hi E(w_hi - d)   for all d.
Starting from the box these rules determine E at every point, so a map that
meets all of them for random u on every axis shape is the closure.  A wrong
mirror index or a sign flipped at one face fails them.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2507_18282_gb300", "csrc")


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("needs g++")
    exe = str(tmp_path_factory.mktemp("bc") / "bc_ext")
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-D__host__=", "-D__device__=", "-D__forceinline__=inline",
                           "-I", CSRC, os.path.join(HERE, "native", "bc_ext.cpp"), "-o", exe])
    rows = np.loadtxt(subprocess.check_output([exe]).decode().splitlines(), dtype=np.int64)
    return rows


def test_32_and_64_bit_indices_agree(table):
    assert np.array_equal(table[:, 3], table[:, 5]) and np.array_equal(table[:, 4], table[:, 6])


@pytest.mark.parametrize("code", [0, 1, 2, 3])
def test_extension_meets_its_definition(table, code):
    rng = np.random.default_rng(7 + code)
    lo_neu, hi_neu = bool(code & 1), bool(code & 2)
    s_lo, s_hi = (1 if lo_neu else -1), (1 if hi_neu else -1)
    rows = table[table[:, 0] == code]
    for n in np.unique(rows[:, 1]):
        r = rows[rows[:, 1] == n]
        p, idx, sgn = r[:, 2], r[:, 3], r[:, 4]
        u = rng.standard_normal(n) + 3.0  # nonzero values, distinct from their negatives
        E = {int(pp): (0.0 if ii < 0 else float(ss * u[ii])) for pp, ii, ss in zip(p, idx, sgn)}
        assert all(s in (-1, 0, 1) for s in sgn)
        for k in range(n):
            assert E[k] == u[k]
        w_lo = 0 if lo_neu else -1
        w_hi = n - 1 if hi_neu else n
        if not lo_neu:
            assert E[-1] == 0.0
        if not hi_neu:
            assert E[n] == 0.0
        pmin, pmax = int(p.min()), int(p.max())
        for d in range(0, pmax - pmin + 1):
            a, b = w_lo - d, w_lo + d
            if a in E and b in E:
                assert E[a] == s_lo * E[b], (n, d, "lower")
            a, b = w_hi + d, w_hi - d
            if a in E and b in E:
                assert E[a] == s_hi * E[b], (n, d, "upper")
        # the reflections reach every listed point from the box: none is left
        # undetermined (a map returning a wall for a non-wall point fails here)
        walls = {w for w, neu in ((w_lo, lo_neu), (w_hi, hi_neu)) if not neu}
        period = 2 * (w_hi - w_lo)
        for pp in E:
            if (pp - w_lo) % period + w_lo not in walls:
                assert E[pp] != 0.0, (n, pp)
