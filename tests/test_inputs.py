"""The seeded input generators (ew_inputs.py), which both the CUDA path and the
oracle receive their buffers from (no GPU).

SplitMix64 is pinned to the test vectors of its published reference
implementation (Steele, Lea, Flood, OOPSLA 2014; the C reference by Vigna,
state advanced by the golden gamma before each output): for seed 0 the first
outputs are 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, and for
seed 1234567 they are 6457827717110365317, 3203168211198807973,
9817491932198370423.  The library's device generator (k_splitmix_uniform)
implements the same definition and is compared with this one on the GPU.
"""
import math

import numpy as np

import ew_inputs as I


def test_splitmix64_reference_vectors():
    assert [int(x) for x in I.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x) for x in I.splitmix64(1234567, 3)] == [6457827717110365317, 3203168211198807973,
                                                          9817491932198370423]


def test_offsets_continue_the_same_stream():
    a = I.splitmix64(I.BASE_SEED, 1000)
    assert np.array_equal(I.splitmix64(I.BASE_SEED, 300, offset=700), a[700:])
    assert np.array_equal(I.uniform_pm1(I.BASE_SEED, 10, offset=5), I.uniform_pm1(I.BASE_SEED, 15)[5:])


def test_uniform_draws_cover_the_interval():
    u = I.uniform_pm1(I.BASE_SEED + 1, 1 << 20)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 5.0 / math.sqrt(3.0 * len(u))    # 5 sigma of the mean of U[-1, 1)
    assert abs(np.mean(u * u) - 1.0 / 3.0) < 5e-3
    # the 53-bit mapping: every value is a multiple of 2^-52 on [-1, 1)
    assert np.all(np.ldexp(u + 1.0, 52) == np.round(np.ldexp(u + 1.0, 52)))


def test_start_block_columns_are_consecutive_draws():
    size, nvec = 37, 4
    X = I.start_block(11, size, nvec)
    assert X.shape == (size, nvec)
    flat = I.uniform_pm1(11, size * nvec)
    for j in range(nvec):
        assert np.array_equal(X[:, j], flat[j * size:(j + 1) * size])


def test_batched_boxes_follow_the_stated_recipe():
    boxes = I.batched_boxes(I.BASE_SEED + 4)
    assert len(boxes) == 64
    ns = np.array([b["n"][0] for b in boxes])
    assert all(b["n"][0] == b["n"][1] for b in boxes)
    assert ns.min() >= 255 and ns.max() <= 2047
    assert all(0.5 <= L <= 2.0 for b in boxes for L in b["length"])
    assert all(10.0 <= b["omega"] <= 200.0 for b in boxes)
    # log-uniform sizes: the median sits near the geometric mean of the range
    assert abs(math.log(np.median(ns)) - 0.5 * (math.log(255) + math.log(2047))) < 0.5


def test_mapped_vertices_keep_the_boundary_on_the_square():
    xy = I.mapped_vertices(30, 20, "square_warp", eps=0.1)
    assert xy.shape == (22, 32, 2)
    x, y = xy[..., 0], xy[..., 1]
    assert np.allclose(x[:, 0], 0.0) and np.allclose(x[:, -1], 1.0)
    assert np.allclose(y[0, :], 0.0) and np.allclose(y[-1, :], 1.0)
    rb = I.mapped_vertices(5, 4, "rotated_box", theta=0.0, lx=2.0, ly=3.0)
    assert np.allclose(rb[-1, -1], (2.0, 3.0))
