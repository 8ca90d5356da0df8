"""Pin of one multigrid cycle of the oracle (eq. impMatrix: M = I - a L_h,
a = dt^2/2) against the cycle assembled here from dense matrices.

Nothing below calls the oracle's stencil, transfer or smoothing code:
  - M on every level is Q diag(1 + a lambda_k^2) Q^T with Q the orthonormal
    tensor sine basis and lambda_k^2 the closed-form discrete eigenvalues of
    the order-2 / order-4 Laplacian with the odd-reflection closure (the sine
    modes are its exact eigenvectors, so this is M itself);
  - restriction: full weighting, the tensor product of the 1D weights
    (1/4, 1/2, 1/4) around fine point 2I + 1 of coarse point I;
  - prolongation: linear interpolation, coarse I onto fine 2I + 1 with weight 1
    and onto the even neighbours 2I, 2I + 2 with weight 1/2 (zero beyond the
    box);
  - the coarsest level solved exactly (dense solve), levels n -> (n - 1)/2
    while every axis is odd and >= 5;
  - damped Jacobi with the constant diagonal D (M's diagonal at a point two
    or more points from every wall), or red-black Gauss-Seidel (points with
    i + j + k even first).
A wrong restriction or interpolation weight, a transposed transfer, a
missing smoothing sweep or a wrong diagonal changes the cycle's output far
beyond the tolerance (the coarsest solve of the oracle is CG to 1e-14)."""
import numpy as np
import pytest

from oracle import oracle as O

TOL = 1e-11


def _axis_basis(n):
    j = np.arange(1, n + 1)[:, None]
    k = np.arange(1, n + 1)[None, :]
    return np.sqrt(2.0 / (n + 1)) * np.sin(np.pi * j * k / (n + 1))


def _axis_symbol(n, h, order):
    s = np.sin(np.arange(1, n + 1) * np.pi / (2 * (n + 1))) ** 2
    return 4.0 / h ** 2 * (s + s * s / 3.0 if order == 4 else s)


def _kron_x_fastest(mats):
    """Kronecker product for vectors with axis 0 (x) fastest: Q_z (x) Q_y (x) Q_x."""
    out = np.ones((1, 1))
    for m in reversed(mats):
        out = np.kron(out, m)
    return out


def _dense_M(n, h, order, a):
    Q = _kron_x_fastest([_axis_basis(m) for m in n])
    lam2 = np.zeros(1)
    for m, hh in zip(n, h):      # eigenvalue of mode (kx, ky, kz), x fastest
        lam2 = (lam2[None, :] + _axis_symbol(m, hh, order)[:, None]).reshape(-1)
    return (Q * (1.0 + a * lam2)[None, :]) @ Q.T


def _restrict_1d(nf):
    nc = (nf - 1) // 2
    R = np.zeros((nc, nf))
    for I in range(nc):
        R[I, 2 * I], R[I, 2 * I + 1], R[I, 2 * I + 2] = 0.25, 0.5, 0.25
    return R


def _prolong_1d(nf):
    nc = (nf - 1) // 2
    P = np.zeros((nf, nc))
    for I in range(nc):
        P[2 * I + 1, I] = 1.0
        P[2 * I, I] += 0.5
        P[2 * I + 2, I] += 0.5
    return P


def _levels(n, h):
    lv = [(tuple(n), tuple(h))]
    while all(m >= 5 and m % 2 == 1 for m in lv[-1][0]):
        m, hh = lv[-1]
        lv.append((tuple((x - 1) // 2 for x in m), tuple(2 * y for y in hh)))
    return lv


def _interior_diag(M, n):
    idx = [min(2, m // 2) for m in n]  # a point two from every wall where the axis allows it
    q = 0
    for a in reversed(range(len(n))):
        q = q * n[a] + idx[a]
    return M[q, q]


def _colour_masks(n, order):
    """Gauss-Seidel colours: (i + j + k) mod 2 at second order, mod 3 at
    fourth order (points flattened x fastest)."""
    grids = np.meshgrid(*[np.arange(m) for m in reversed(n)], indexing="ij")
    ncol = 2 if order == 2 else 3
    col = sum(grids).reshape(-1) % ncol
    return [col == c for c in range(ncol)]


class DenseCycle:
    def __init__(self, n, h, order, a, wJ, red_black):
        self.lv = _levels(n, h)
        self.M = [_dense_M(m, hh, order, a) for m, hh in self.lv]
        self.R = [_kron_x_fastest([_restrict_1d(x) for x in m]) for m, _ in self.lv[:-1]]
        self.P = [_kron_x_fastest([_prolong_1d(x) for x in m]) for m, _ in self.lv[:-1]]
        self.D = [_interior_diag(M, m) for M, (m, _) in zip(self.M, self.lv)]
        self.col = [_colour_masks(m, order) for m, _ in self.lv]
        self.wJ, self.red_black = wJ, red_black

    def smooth(self, L, b, x, nu):
        M, D = self.M[L], self.D[L]
        for _ in range(nu):
            if self.red_black:
                for mask in self.col[L]:
                    x = x + np.where(mask, (b - M @ x) / D, 0.0)
            else:
                x = x + self.wJ * (b - M @ x) / D
        return x

    def cycle(self, L, b, x, nu1, nu2):
        if L == len(self.lv) - 1:
            return np.linalg.solve(self.M[L], b)
        x = self.smooth(L, b, x, nu1)
        ec = self.cycle(L + 1, self.R[L] @ (b - self.M[L] @ x), np.zeros(self.M[L + 1].shape[0]), nu1, nu2)
        x = x + self.P[L] @ ec
        return self.smooth(L, b, x, nu2)


CASES = [
    # (n, length, order, red_black)
    ((7, 7, 7), (1.0, 1.0, 1.0), 2, False),
    ((7, 7, 7), (1.0, 0.8, 1.2), 4, False),
    ((15, 31), (1.0, 1.7), 2, False),          # three levels, anisotropic h
    ((15, 31), (1.0, 1.7), 4, False),
    ((15, 15), (1.0, 1.0), 2, True),
    ((7, 7, 7), (1.0, 1.0, 1.0), 2, True),
    ((15, 31), (1.0, 1.7), 4, True),           # three colours
    ((7, 15, 7), (1.0, 0.8, 1.2), 4, True),
]


@pytest.mark.parametrize("n,length,order,red_black", CASES)
@pytest.mark.parametrize("nu1,nu2", [(1, 0), (0, 1), (2, 1)])
def test_one_cycle_equals_the_dense_cycle(n, length, order, red_black, nu1, nu2):
    g = O.Grid(n, length, order)
    a = 0.01 * min(g.h) ** 2 * 64
    rng = np.random.default_rng(11)
    b = rng.uniform(-1, 1, g.size)
    x0 = rng.uniform(-1, 1, g.size)
    ref = DenseCycle(n, g.h, order, a, 0.8, red_black)
    want = ref.cycle(0, b, x0.copy(), nu1, nu2)
    got, hist = O.mg_solve(g, a, b, x0=x0, nu1=nu1, nu2=nu2, wJ=0.8, ncycles=1, red_black=red_black)
    assert np.max(np.abs(got - want)) <= TOL * np.max(np.abs(want))
    # the residual history: before and after the cycle
    assert hist[0] == pytest.approx(np.linalg.norm(b - ref.M[0] @ x0), rel=1e-12)
    assert hist[1] == pytest.approx(np.linalg.norm(b - ref.M[0] @ want), rel=1e-8, abs=1e-13)


def test_two_cycles_carry_the_iterate():
    n, length, order = (15, 31), (1.0, 1.7), 4
    g = O.Grid(n, length, order)
    a = 0.3 * min(g.h) ** 2
    rng = np.random.default_rng(12)
    b = rng.uniform(-1, 1, g.size)
    ref = DenseCycle(n, g.h, order, a, 0.8, False)
    want = ref.cycle(0, b, np.zeros(g.size), 2, 2)
    want = ref.cycle(0, b, want, 2, 2)
    got, _ = O.mg_solve(g, a, b, nu1=2, nu2=2, wJ=0.8, ncycles=2)
    assert np.max(np.abs(got - want)) <= TOL * np.max(np.abs(want))


def test_dense_M_is_the_oracle_operator():
    """The dense M built from the sine basis is the operator the oracle applies
    (both orders; the sine modes are exact eigenvectors of the closure)."""
    for n, length, order in [((7, 7, 7), (1.0, 0.8, 1.2), 4), ((15, 31), (1.0, 1.7), 2)]:
        g = O.Grid(n, length, order)
        a = 0.02
        M = _dense_M(n, g.h, order, a)
        x = np.random.default_rng(3).uniform(-1, 1, g.size)
        assert np.max(np.abs(O.apply_M(g, a, x) - M @ x)) <= 1e-11 * np.max(np.abs(M @ x))


@pytest.mark.parametrize("n,order", [((15, 31), 2), ((9, 7, 11), 2), ((15, 31), 4), ((9, 7, 11), 4)])
def test_colours_do_not_couple(n, order):
    """No entry of M joins two distinct points of one colour, so updating a
    colour point by point (the oracle) equals updating it at once (the dense
    cycle, and the GPU's one launch per colour)."""
    g = O.Grid(n, tuple(1.0 for _ in n), order)
    M = _dense_M(n, g.h, order, 0.3)
    for mask in _colour_masks(n, order):
        blk = M[np.ix_(mask, mask)]
        off = blk - np.diag(np.diag(blk))
        assert np.max(np.abs(off)) <= 1e-12 * np.max(np.abs(M))
    # and the colouring is not vacuous: M does join points of different colours
    masks = _colour_masks(n, order)
    assert np.max(np.abs(M[np.ix_(masks[0], masks[1])])) > 0.1 * np.max(np.abs(M))
