"""The double-FP32 pair arithmetic of the FP64-accuracy wave-solves
(paper_2507_18282_gb300/csrc/ew_dd.cuh), compiled for the host and checked
against long double (no GPU): each result is an unevaluated sum hi + lo with
|lo| <= ulp(hi)/2, and each operation's error is a few 2^-48 of its operands
(addition and multiply-add bounded relative to |x| + |y|, product relative to
|x y|, conversion from FP64 relative to the value)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2507_18282_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_pair_operations_meet_their_bounds(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "pair_arith")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-D__host__=", "-D__device__=",
                           "-D__forceinline__=inline", "-D__align__(x)=alignas(x)", "-I", CSRC, "-I", inc,
                           os.path.join(HERE, "native", "pair_arith.cpp"), "-o", exe])
    conv, add, mul, fma, canc, nonoverlap = map(float, subprocess.check_output([exe]).split())
    u = 2.0 ** -48
    assert conv <= 0.51 * u      # nearest pair to an FP64 value
    assert add <= 4 * u          # two_sum + trailing parts + renormalisation
    assert mul <= 5 * u
    assert fma <= 8 * u
    assert canc <= 2 * u         # near-total cancellation stays operand-bounded
    assert nonoverlap <= 1.0     # results are renormalised
