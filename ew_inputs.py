"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the EigenWave method: it only draws
numbers.  Both the CUDA path and the CPU oracle receive the buffers made here.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): the i-th draw of stream `seed` is
mix(seed + (i + 1) * 0x9E3779B97F4A7C15) with the published 64-bit finaliser,
mapped to a double u = (z >> 11) * 2^-53 in [0, 1).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

#: base seed of the workload presets; preset i uses BASE_SEED + i
BASE_SEED = 2507182820


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` raw 64-bit draws of stream `seed`, starting at draw `offset`."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Start vectors: uniform on [-1, 1) on the active (interior) points, FP64."""
    return 2.0 * uniform01(seed, count, offset) - 1.0


def start_block(seed: int, size: int, nvec: int) -> np.ndarray:
    """`nvec` start vectors of length `size`, column j from draws j*size...(j+1)*size-1."""
    return uniform_pm1(seed, size * nvec).reshape(nvec, size).T.copy()


def batched_boxes(seed: int, count: int = 64, n_min: int = 255, n_max: int = 2047,
                  len_min: float = 0.5, len_max: float = 2.0, w_min: float = 10.0,
                  w_max: float = 200.0):
    """Uneven 2D Dirichlet boxes for the batched workload.

    Problem p takes draws 4p..4p+3 in this order: side lengths Lx, Ly ~ U[0.5, 2],
    grid size n ~ log-uniform integer in [n_min, n_max] (an n x n grid, so
    h_x != h_y in general), target omega ~ U[10, 200]."""
    u = uniform01(seed, 4 * count).reshape(count, 4)
    out = []
    for p in range(count):
        lx = len_min + (len_max - len_min) * u[p, 0]
        ly = len_min + (len_max - len_min) * u[p, 1]
        n = int(round(math.exp(math.log(n_min) + u[p, 2] * (math.log(n_max) - math.log(n_min)))))
        n = min(max(n, n_min), n_max)
        w = w_min + (w_max - w_min) * u[p, 3]
        out.append(dict(n=(n, n), length=(lx, ly), omega=w))
    return out


def learned_init(seed: int, scale: float = 0.05) -> np.ndarray:
    """Initial learned-smoother weights (2 x 8 x 27), uniform in [-scale, scale)."""
    return scale * uniform_pm1(seed, 2 * 8 * 27)


# ----------------------------------------------------------------------------
# curvilinear grids (vertex coordinates of a map x = G(r) from the unit square)
# ----------------------------------------------------------------------------

def mapped_vertices(n1: int, n2: int, kind: str = "square_warp", eps: float = 0.1, theta: float = 0.3,
                    lx: float = 1.0, ly: float = 1.0) -> np.ndarray:
    """Vertex coordinates, shape (n2 + 2, n1 + 2, 2) with the r1 index fastest,
    boundary vertices included, of one of the test geometries:
      square_warp   x = r + eps sin(pi r) cos(pi s), y = s + eps sin(pi s) cos(pi r):
                    a smooth map of the unit square onto itself (boundary onto
                    boundary), so the continuous eigenvalues are pi^2 (k^2 + l^2)
      rotated_box   the box [0, lx] x [0, ly] rotated by theta about the origin
    Geometry only: nothing here computes the method."""
    r = np.linspace(0.0, 1.0, n1 + 2)
    s = np.linspace(0.0, 1.0, n2 + 2)
    R, S = np.meshgrid(r, s)  # (n2 + 2, n1 + 2), r fastest
    if kind == "square_warp":
        x = R + eps * np.sin(np.pi * R) * np.cos(np.pi * S)
        y = S + eps * np.sin(np.pi * S) * np.cos(np.pi * R)
    elif kind == "rotated_box":
        c, sn = np.cos(theta), np.sin(theta)
        x = c * lx * R - sn * ly * S
        y = sn * lx * R + c * ly * S
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(np.stack([x, y], axis=-1))
