"""FP64 CPU oracle for the EigenWave filter operator (arXiv 2507.18282).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library under ``paper_2507_18282_gb300/``: the grid stencils and
time stepping live in ``ew_oracle.c`` (plain loops, no FMA contraction), the
parameter math, closed forms and the Krylov eigen-solver are written out here
in numpy.  Library primitives used as single steps: ``numpy.linalg.eigh``
(small dense symmetric eigenproblem), ``numpy.linalg.qr`` and
``scipy.fft.dstn`` (exact sine transform on boxes).

Each function names the passage of the paper it follows.  Parity pins (what
keeps this oracle honest) live in ``tests/test_oracle_*.py``.  Functions with
no pin say "parity unpinned" in their docstring.
"""
from __future__ import annotations

import ctypes
import math
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build", platform.machine())
_SO = os.path.join(_BUILD, "libew_oracle.so")
_SOURCES = ["ew_oracle.c", "ew_oracle_mg.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp] + srcs + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(ctypes.c_long)
            i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
            ip = ctypes.POINTER(ctypes.c_int)
            lib.og_apply_L.argtypes = [i, lp, dp, i, ip, dp, dp]
            lib.og_apply_M.argtypes = [i, lp, dp, i, d, dp, dp]
            lib.og_filter_explicit.argtypes = [i, lp, dp, i, ip, l, d, dp, dp, dp]
            lib.og_filter_implicit.argtypes = [i, lp, dp, i, l, d, dp, dp, dp, d]
            lib.og_cg_solve_M.argtypes = [i, lp, dp, i, d, dp, dp, d, i]
            lib.og_mg_solve.argtypes = [i, lp, dp, i, d, dp, dp, i, i, d, i, dp, i, dp, i]
            lib.og_mapped_apply_L.argtypes = [l, l, dp, dp, dp]
            lib.og_mapped_jacobian.argtypes = [l, l, dp, dp]
            lib.og_mapped_filter_explicit.argtypes = [l, l, dp, l, d, dp, dp, dp]
            lib.og_conv_net_forward.argtypes = [lp, dp, dp, dp, dp]
            lib.og_conv_net_backward.argtypes = [lp, dp, dp, dp, dp, dp, dp]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Grid:
    """Cartesian box (eq. eigBVPdiscrete) with homogeneous Dirichlet faces or
    Neumann faces (the paper's symmetry-plane condition).

    ``n`` = interior points per axis, ``length`` = box side lengths,
    h_i = length_i / (n_i + 1); ``bc`` = None (all Dirichlet) or 2 dim face
    kinds "D" / "N" in the order -x, +x, -y, +y[, -z, +z].  A Neumann face's
    wall points are active, so axis i has ``nact[i]`` = n_i + (its Neumann
    faces) active points.  Vectors hold active points, x fastest (Algorithm
    matVec; Note 1 of the Arnoldi section)."""

    def __init__(self, n, length, order, bc=None):
        self.dim = len(n)
        assert self.dim in (2, 3) and order in (2, 4)
        self.n = tuple(int(v) for v in n)
        self.length = tuple(float(v) for v in length)
        self.order = int(order)
        self.bc = tuple("D" for _ in range(2 * self.dim)) if bc is None else tuple(bc)
        assert len(self.bc) == 2 * self.dim and all(f in ("D", "N") for f in self.bc)
        self.h = tuple(L / (m + 1) for L, m in zip(self.length, self.n))
        self.nact = tuple(m + (self.bc[2 * a] == "N") + (self.bc[2 * a + 1] == "N")
                          for a, m in enumerate(self.n))
        self.size = int(np.prod(self.nact))
        self.neumann = "N" in self.bc
        self._n3 = (ctypes.c_long * 3)(*(list(self.nact) + [1] * (3 - self.dim)))
        self._h3 = (ctypes.c_double * 3)(*(list(self.h) + [1.0] * (3 - self.dim)))
        self._bc6 = (ctypes.c_int * 6)(*([int(f == "N") for f in self.bc] + [0] * (6 - 2 * self.dim)))

    @property
    def shape(self):
        """numpy shape of a grid function with x fastest."""
        return tuple(reversed(self.nact))

    def dirichlet_only(self):
        assert not self.neumann, "this oracle routine takes Dirichlet boxes only"


# ----------------------------------------------------------------------------
# grid operators (C)
# ----------------------------------------------------------------------------

def apply_L(g: Grid, u):
    """L_h u, the order-p centred Laplacian with Dirichlet closure (eq. eigBVPdiscrete)."""
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    out = np.empty_like(u)
    rc = _load().og_apply_L(g.dim, g._n3, g._h3, g.order, g._bc6, _dp(u), _dp(out))
    assert rc == 0
    return out


def apply_M(g: Grid, a, x):
    """M x = (I - a L_h) x with a = dt^2/2 (eq. impMatrix)."""
    g.dirichlet_only()
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    out = np.empty_like(x)
    rc = _load().og_apply_M(g.dim, g._n3, g._h3, g.order, float(a), _dp(x), _dp(out))
    assert rc == 0
    return out


def cg_solve_M(g: Grid, a, b, tol=1e-14, maxit=100000):
    """Solve M x = b by conjugate gradients (M symmetric positive definite, eq. impMatrix)."""
    g.dirichlet_only()
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    x = np.empty_like(b)
    it = _load().og_cg_solve_M(g.dim, g._n3, g._h3, g.order, float(a), _dp(b), _dp(x),
                               float(tol), int(maxit))
    assert it >= 0, "CG did not converge"
    return x


# ----------------------------------------------------------------------------
# a1: filter parameters
# ----------------------------------------------------------------------------

def spectral_radius_bound(g: Grid):
    """Largest eigenvalue of -L_h on the box: the mode symbol at sin^2 = 1
    (the CFL limit of reading c2 takes dt_max = 2 / sqrt of it).

    Order 2: 4 sum 1/h_i^2.  Order 4: (4 + 4/3) sum 1/h_i^2 (1D symbol of the
    (-1, 16, -30, 16, -1)/12 stencil is 4 s + (4/3) s^2, s = sin^2(theta/2))."""
    inv = sum(1.0 / (h * h) for h in g.h)
    return (4.0 if g.order == 2 else 16.0 / 3.0) * inv


def steps_per_period_cfl(g: Grid, omega, cfl):
    """Explicit steps per period: the paper defers the CFL rule to its WaveHoltz
    references, so this follows the standard leapfrog stability limit
    dt <= 2 / sqrt(rho(-L_h)) scaled by ``cfl`` (reading recorded in the design
    notes)."""
    dt_max = 2.0 / math.sqrt(spectral_radius_bound(g))
    period = 2.0 * math.pi / omega
    return int(math.ceil(period / (cfl * dt_max) - 1e-12))


def adjusted_omega(omega, n_its):
    """omega~ of eq. adjustedOmega: the target that makes the time-corrected
    implicit filter peak at lambda = omega (needs n_its > 4)."""
    s2 = math.sin(math.pi / n_its) ** 2
    return omega * math.pi / n_its * math.sqrt((1.0 - 2.0 * s2) / s2)


def filter_params(omega, num_periods, steps_per_period, adjust=False):
    """Host parameters of one wave-solve (Section 'Discrete approximations').

    T_f = N_p 2 pi / omega, N_t = N_p * steps_per_period, dt = T_f / N_t,
    alpha_d = tan(omega dt/2) / tan(omega dt)            (eq. alphad),
    c_n = (2/T_f) sigma_n (cos(omega t^n) - alpha_d/2)    (eq. filterQuadrature)
    with the trapezoid weights sigma_0 = sigma_Nt = dt/2, else dt.
    With ``adjust`` omega is replaced by omega~ (eq. adjustedOmega) everywhere."""
    w = adjusted_omega(omega, steps_per_period) if adjust else float(omega)
    Tf = num_periods * 2.0 * math.pi / w
    Nt = int(num_periods) * int(steps_per_period)
    dt = Tf / Nt
    alpha_d = math.tan(w * dt / 2.0) / math.tan(w * dt)
    n = np.arange(Nt + 1, dtype=np.float64)
    sigma = np.full(Nt + 1, dt)
    sigma[0] = sigma[-1] = dt / 2.0
    c = (2.0 / Tf) * sigma * (np.cos(w * n * dt) - alpha_d / 2.0)
    return dict(omega=w, Tf=Tf, Nt=Nt, dt=dt, alpha_d=alpha_d, c=c)


# ----------------------------------------------------------------------------
# a2-a5: one wave-solve = one application of S (Algorithm matVec)
# ----------------------------------------------------------------------------

def filter_explicit(g: Grid, prm, v):
    """S v with explicit leapfrog (eqs. explicitScheme, explicitStep1, filterQuadrature)."""
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    c = np.ascontiguousarray(prm["c"], dtype=np.float64)
    out = np.empty_like(v)
    rc = _load().og_filter_explicit(g.dim, g._n3, g._h3, g.order, g._bc6, int(prm["Nt"]),
                                    float(prm["dt"]), _dp(c), _dp(v), _dp(out))
    assert rc == 0
    return out


def filter_implicit(g: Grid, prm, v, tol=1e-14):
    """S v with the implicit trapezoidal scheme, every M-solve done by CG to
    ``tol`` (eqs. implicitScheme, impMatrix, implicitStep1, filterQuadrature)."""
    g.dirichlet_only()
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    c = np.ascontiguousarray(prm["c"], dtype=np.float64)
    out = np.empty_like(v)
    rc = _load().og_filter_implicit(g.dim, g._n3, g._h3, g.order, int(prm["Nt"]),
                                    float(prm["dt"]), _dp(c), _dp(v), _dp(out), float(tol))
    assert rc == 0
    return out


def filter_apply(g: Grid, prm, v, scheme="explicit"):
    """S v (Algorithm matVec) with the explicit or the implicit scheme."""
    return filter_explicit(g, prm, v) if scheme == "explicit" else filter_implicit(g, prm, v)


# ----------------------------------------------------------------------------
# closed forms on boxes (pins; Section 'discrete analysis')
# ----------------------------------------------------------------------------

def mode_indices(g: Grid):
    """All multi-indices k (1-based per axis) in vector order of the DST."""
    g.dirichlet_only()
    axes = [np.arange(1, m + 1) for m in g.n]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def lambda2_closed_form(g: Grid, k):
    """Discrete Dirichlet eigenvalue lambda_h^2 of -L_h for sine mode k: the
    true discrete eigenvalues of eq. eigBVPdiscrete on a box (Section
    "Accuracy of eigenpairs"), in closed form.

    With s_i = sin^2(k_i pi / (2 (n_i + 1))):  order 2: sum 4 s_i / h_i^2;
    order 4 (odd-reflection closure): sum 4 (s_i + s_i^2 / 3) / h_i^2."""
    k = np.atleast_2d(np.asarray(k, dtype=np.float64))
    lam2 = np.zeros(k.shape[0])
    for a in range(g.dim):
        s = np.sin(k[:, a] * math.pi / (2.0 * (g.n[a] + 1))) ** 2
        sym = 4.0 * s if g.order == 2 else 4.0 * (s + s * s / 3.0)
        lam2 += sym / (g.h[a] ** 2)
    return lam2


def sine_mode(g: Grid, k):
    """Tensor sine mode phi_k(x_i) = prod_a sin(k_a pi (i_a + 1) / (n_a + 1)), as an active vector."""
    g.dirichlet_only()
    vecs = [np.sin(k[a] * math.pi * np.arange(1, g.n[a] + 1) / (g.n[a] + 1)) for a in range(g.dim)]
    out = vecs[0]
    for a in range(1, g.dim):
        out = np.multiply.outer(vecs[a], out)
    return np.ascontiguousarray(out.reshape(-1))


def lambda_tilde_explicit(lam, dt):
    """Time-corrected frequency of leapfrog, eq. discreteExplicitLambdaTilde."""
    return (2.0 / dt) * np.arcsin(np.asarray(lam) * dt / 2.0)


def lambda_tilde_implicit(lam, dt):
    """Time-corrected frequency of the implicit scheme, eq. discreteCorr."""
    lam = np.asarray(lam)
    return (2.0 / dt) * np.arcsin(0.5 * lam * dt / np.sqrt(1.0 + 0.5 * (lam * dt) ** 2))


def beta_d(lam_tilde, prm):
    """Discrete filter function eq. betad: sum_n c_n cos(lam~ t^n)."""
    t = np.arange(prm["Nt"] + 1) * prm["dt"]
    lt = np.atleast_1d(np.asarray(lam_tilde, dtype=np.float64))
    return np.cos(np.outer(lt, t)) @ prm["c"]


def beta_tilde(lam, prm, scheme="explicit"):
    """Time-corrected discrete filter eq. correctedBeta for spatial eigenvalue lam."""
    lt = lambda_tilde_explicit(lam, prm["dt"]) if scheme == "explicit" else \
        lambda_tilde_implicit(lam, prm["dt"])
    return beta_d(lt, prm)


def beta_continuous(lam, omega, Tf):
    """Continuous filter, sinc form eq. filterThreeSincs (sinc x = sin x / x)."""
    def sinc(x):
        x = np.asarray(x, dtype=np.float64)
        return np.where(np.abs(x) < 1e-300, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))
    lam = np.asarray(lam, dtype=np.float64)
    return sinc((omega - lam) * Tf) + sinc((omega + lam) * Tf) - 0.5 * sinc(lam * Tf)


def dst(g: Grid, v):
    """Orthonormal DST-I over every axis: coefficients of v in the normalised sine modes."""
    g.dirichlet_only()
    import scipy.fft
    return scipy.fft.dstn(np.asarray(v, dtype=np.float64).reshape(g.shape), type=1,
                          norm="ortho").reshape(-1)


def idst(g: Grid, vhat):
    """Inverse of ``dst``: the active vector with sine-mode coefficients vhat."""
    import scipy.fft
    return scipy.fft.idstn(np.asarray(vhat, dtype=np.float64).reshape(g.shape), type=1,
                           norm="ortho").reshape(-1)


def spectrum(g: Grid):
    """lambda_h^2 of every sine mode, in DST coefficient order (x fastest)."""
    g.dirichlet_only()
    axes = [np.arange(1, m + 1) for m in reversed(g.n)]
    mesh = np.meshgrid(*axes, indexing="ij")   # slowest axis first
    k = np.stack([m.reshape(-1) for m in reversed(mesh)], axis=1)  # columns kx, ky, (kz)
    return lambda2_closed_form(g, k), k


def filter_closed_form(g: Grid, prm, v, power=1, scheme="explicit"):
    """S^power v on a box, computed in the sine basis: S is diagonal there with
    entries beta~_d(lambda_k) (Theorem 'Eigenvalues of the EigenWave operator',
    discrete form eq. discreteBeta).  Boxes with Neumann faces use the
    tensor sine / cosine modes of ``axis_modes``."""
    if g.neumann:
        return modes_closed_form(g, v, lambda lam2: beta_tilde(np.sqrt(lam2), prm, scheme) ** power)
    lam2, _ = spectrum(g)
    b = beta_tilde(np.sqrt(lam2), prm, scheme)
    return idst(g, (b ** power) * dst(g, v))


def axis_modes(g: Grid, a):
    """Exact eigenvectors of L_h along axis a (Section 'discrete analysis':
    the closure is a reflection about the wall point, so the modes of the
    infinite grid that obey it are eigenvectors of the box), as the columns of
    a matrix over the axis's active points, with their angles theta.  With
    M = n_a + 1 and the vertex index j (walls at j = 0 and j = M):
      D-D  sin(theta j), theta = k pi / M,         k = 1 .. M-1, j = 1 .. M-1
      N-N  cos(theta j), theta = k pi / M,         k = 0 .. M,   j = 0 .. M
      N-D  cos(theta j), theta = (k - 1/2) pi / M, k = 1 .. M,   j = 0 .. M-1
      D-N  sin(theta j), theta = (k - 1/2) pi / M, k = 1 .. M,   j = 1 .. M
    (odd about a Dirichlet wall, even about a Neumann wall)."""
    lo, hi = g.bc[2 * a], g.bc[2 * a + 1]
    M = g.n[a] + 1
    if lo == "D" and hi == "D":
        th, j, f = np.arange(1, M) * math.pi / M, np.arange(1, M), np.sin
    elif lo == "N" and hi == "N":
        th, j, f = np.arange(0, M + 1) * math.pi / M, np.arange(0, M + 1), np.cos
    elif lo == "N":
        th, j, f = (np.arange(1, M + 1) - 0.5) * math.pi / M, np.arange(0, M), np.cos
    else:
        th, j, f = (np.arange(1, M + 1) - 0.5) * math.pi / M, np.arange(1, M + 1), np.sin
    return th, f(np.outer(j, th))


def axis_symbol(g: Grid, a, theta):
    """1D eigenvalue of -L_h along axis a for angle theta, s = sin^2(theta / 2):
    order 2: 4 s / h^2; order 4: 4 (s + s^2 / 3) / h^2 (the symbol of
    (-1, 16, -30, 16, -1) / 12)."""
    s = np.sin(0.5 * np.asarray(theta)) ** 2
    return (4.0 * s if g.order == 2 else 4.0 * (s + s * s / 3.0)) / (g.h[a] ** 2)


def spectrum_modes(g: Grid):
    """lambda_h^2 of every tensor mode of ``axis_modes`` (any faces), in mode
    order with the x index fastest."""
    lam2 = np.zeros(1)
    for a in range(g.dim):
        th, _ = axis_modes(g, a)
        lam2 = np.add.outer(axis_symbol(g, a, th), lam2)   # new axis slowest
    return lam2.reshape(-1)


def modes_closed_form(g: Grid, v, fn):
    """Apply the function fn(lambda^2) of L_h to v exactly: expand v in the
    tensor modes of ``axis_modes`` (a solve per axis), scale each coefficient,
    sum the modes back."""
    mats = [axis_modes(g, a)[1] for a in range(g.dim)]
    x = np.asarray(v, dtype=np.float64).reshape(g.shape)   # (z,) y, x
    for a in range(g.dim):
        ax = g.dim - 1 - a
        x = np.moveaxis(np.tensordot(np.linalg.inv(mats[a]), x, axes=([1], [ax])), 0, ax)
    x = x.reshape(-1) * fn(spectrum_modes(g))
    x = x.reshape(g.shape)
    for a in range(g.dim):
        ax = g.dim - 1 - a
        x = np.moveaxis(np.tensordot(mats[a], x, axes=([1], [ax])), 0, ax)
    return x.reshape(-1)


def tensor_mode(g: Grid, k):
    """Tensor mode with 0-based mode indices k = (kx, ky[, kz]) of ``axis_modes``, as an active vector."""
    out = axis_modes(g, 0)[1][:, k[0]]
    for a in range(1, g.dim):
        out = np.multiply.outer(axis_modes(g, a)[1][:, k[a]], out)
    return np.ascontiguousarray(out.reshape(-1))


def trapezoid_weights(g: Grid):
    """Weights of the discrete L_2 inner product on the active points (eq.
    discreteRayleighQuotient): the trapezoid rule, 1/2 per Neumann wall coordinate (all 1 on Dirichlet
    boxes, whose walls are not active).  L_h is symmetric in these weights."""
    w = np.ones(1)
    for a in range(g.dim):
        wa = np.ones(g.nact[a])
        if g.bc[2 * a] == "N":
            wa[0] = 0.5
        if g.bc[2 * a + 1] == "N":
            wa[-1] = 0.5
        w = np.multiply.outer(wa, w)
    return w.reshape(-1)


def implicit_solve_closed_form(g: Grid, a, b):
    """M^{-1} b on a box: divide each sine coefficient by 1 + a lambda^2 (eq. impMatrix)."""
    g.dirichlet_only()
    lam2, _ = spectrum(g)
    return idst(g, dst(g, b) / (1.0 + a * lam2))


# ----------------------------------------------------------------------------
# single curvilinear grid by the mapping method (ew_oracle.c: og_mapped_*)
# ----------------------------------------------------------------------------

class MappedGrid:
    """A 2D curvilinear grid x = G(r) of the unit square (Section "Discrete
    approximations", the mapping method), second order, u = 0 on the boundary
    vertices.  ``n`` = (n1, n2) interior vertices; ``xy`` = vertex coordinates,
    shape (n2 + 2, n1 + 2, 2), r1 index fastest.  Vectors hold the interior
    vertices, r1 fastest."""

    def __init__(self, n, xy):
        self.n = (int(n[0]), int(n[1]))
        self.xy = np.ascontiguousarray(xy, dtype=np.float64)
        assert self.xy.shape == (self.n[1] + 2, self.n[0] + 2, 2)
        self.size = self.n[0] * self.n[1]


def mapped_apply_L(m: MappedGrid, u):
    """L u in the conservative form of the transformed Laplacian (ew_oracle.c)."""
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    out = np.empty_like(u)
    rc = _load().og_mapped_apply_L(m.n[0], m.n[1], _dp(m.xy), _dp(u), _dp(out))
    assert rc == 0, rc
    return out


def mapped_jacobian(m: MappedGrid):
    """J = det(dx/dr) at the active vertices: the weights in which L is symmetric."""
    out = np.empty(m.size)
    rc = _load().og_mapped_jacobian(m.n[0], m.n[1], _dp(m.xy), _dp(out))
    assert rc == 0, rc
    return out


def mapped_filter_explicit(m: MappedGrid, prm, v):
    """S v on the mapped grid with explicit leapfrog (eqs. explicitScheme, explicitStep1, filterQuadrature)."""
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    c = np.ascontiguousarray(prm["c"], dtype=np.float64)
    out = np.empty_like(v)
    rc = _load().og_mapped_filter_explicit(m.n[0], m.n[1], _dp(m.xy), int(prm["Nt"]), float(prm["dt"]),
                                           _dp(c), _dp(v), _dp(out))
    assert rc == 0, rc
    return out


def mapped_rayleigh_lambda(m: MappedGrid, phi):
    """lambda from the Rayleigh quotient in the J-weighted sums (eq. discreteRayleighQuotient)."""
    phi = np.asarray(phi, dtype=np.float64).reshape(-1)
    w = mapped_jacobian(m)
    lam2 = -np.dot(w * phi, mapped_apply_L(m, phi)) / np.dot(w * phi, phi)
    return math.sqrt(max(lam2, 0.0))


# ----------------------------------------------------------------------------
# a8: Rayleigh quotient, residual, accuracy metrics
# ----------------------------------------------------------------------------

def rayleigh_lambda(g: Grid, phi):
    """lambda from the unweighted Rayleigh quotient eq. simpleRayleighQuotient:
    -lambda^2 = sum phi L phi / sum phi^2 over active points; with Neumann
    faces both sums carry the trapezoid weights (eq. discreteRayleighQuotient)."""
    phi = np.asarray(phi, dtype=np.float64).reshape(-1)
    w = trapezoid_weights(g)
    lam2 = -np.dot(w * phi, apply_L(g, phi)) / np.dot(w * phi, phi)
    return math.sqrt(max(lam2, 0.0))


def eig_res(g: Grid, lam, phi):
    """eig-res = ||L V + lambda^2 V||_inf / lambda^2 with ||V||_inf = 1 (accuracy metrics,
    Section 'Numerical results')."""
    phi = np.asarray(phi, dtype=np.float64).reshape(-1)
    phi = phi / np.max(np.abs(phi))
    return float(np.max(np.abs(apply_L(g, phi) + lam * lam * phi)) / (lam * lam))


def eigenspace_distance(v, basis):
    """evect-err for a possibly multiple eigenvalue (accuracy metrics of
    Section "Numerical results": the distance to the closest vector of the
    true discrete eigenspace): max-norm distance from v (scaled to
    ||v||_inf = 1) to its least-squares projection onto span(basis)."""
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    v = v / np.max(np.abs(v))
    B = np.asarray(basis, dtype=np.float64).reshape(len(v), -1)
    coef, *_ = np.linalg.lstsq(B, v, rcond=None)
    return float(np.max(np.abs(v - B @ coef)))


# ----------------------------------------------------------------------------
# a6: multigrid for the implicit systems and the learned smoother (ew_oracle_mg.c)
# ----------------------------------------------------------------------------

NET_WEIGHTS = 2 * 8 * 27   # [W1 (8 x 27) | W2 (8 x 27)], taps (dz, dy, dx), dz slowest


def mg_solve(g: Grid, a, b, x0=None, nu1=2, nu2=2, wJ=0.8, ncycles=1, net=None, red_black=False):
    """``ncycles`` multigrid V(nu1, nu2) cycles on (I - a L_h) x = b (eq. impMatrix).

    The cycle (Jacobi, multi-colour Gauss-Seidel (red-black at order 2, three
    colours at order 4) or learned smoother,
    full weighting, linear interpolation, CG on the coarsest level) is spelled
    out in ew_oracle_mg.c.
    ``net`` is None or an array (levels x NET_WEIGHTS) of learned-smoother
    weights for the finest levels.  Returns (x, residual 2-norm history)."""
    g.dirichlet_only()
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
    hist = np.zeros(ncycles + 1)
    if net is None:
        netp, nl = None, 0
    else:
        net = np.ascontiguousarray(np.atleast_2d(net), dtype=np.float64)
        netp, nl = _dp(net), net.shape[0]
    nlev = _load().og_mg_solve(g.dim, g._n3, g._h3, g.order, float(a), _dp(b), _dp(x),
                               int(nu1), int(nu2), float(wJ), int(ncycles), netp, int(nl),
                               _dp(hist), int(bool(red_black)))
    assert nlev > 0
    return x, hist


def filter_implicit_mg(g: Grid, prm, v, nu1=2, nu2=2, wJ=0.8, ncycles=2, net=None, guess="rhs",
                       return_hist=False):
    """S v with the implicit scheme (eqs. implicitScheme, implicitStep1) where
    every system M y = rhs gets `ncycles` multigrid V-cycles (ew_oracle_mg.c).
    The systems are M W^1 = W^0 and, for n >= 1, M y = 2 W^n with
    y = W^{n+1} + W^{n-1}.  The paper does not state the initial guess:
      guess="rhs"       y = rhs (W^0 for the first system, 2 W^n after);
      guess="previous"  from the third system on, the previous system's
                        solution y_{n-1} = W^n + W^{n-2} (the second system
                        starts from 2 W^1, which is y_0 = W^1 + W^{-1} under
                        the initial condition W^{-1} = W^1).  When that system
                        was solved exactly, M y_{n-1} = 2 W^{n-1}, so the
                        initial residual is 2 (W^n - W^{n-1}), whatever h.
    With ncycles large both tend to filter_implicit.  return_hist: also return
    each system's residual history (before and after each cycle)."""
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    if guess not in ("rhs", "previous"):
        raise ValueError("guess must be 'rhs' or 'previous'")
    a = 0.5 * prm["dt"] ** 2
    c = prm["c"]
    wm = v.copy()
    w0, h = mg_solve(g, a, wm, x0=wm, nu1=nu1, nu2=nu2, wJ=wJ, ncycles=ncycles, net=net)
    hists = [h]
    out = c[0] * wm + c[1] * w0
    y_prev = None
    for n in range(1, prm["Nt"]):
        rhs = 2.0 * w0
        x0 = y_prev if (guess == "previous" and y_prev is not None) else rhs
        y, h = mg_solve(g, a, rhs, x0=x0, nu1=nu1, nu2=nu2, wJ=wJ, ncycles=ncycles, net=net)
        hists.append(h)
        y_prev = y
        wp = y - wm
        wm, w0 = w0, wp
        out = out + c[n + 1] * wp
    return (out, hists) if return_hist else out


def conv_net_forward(n3, w, r):
    """Learned-smoother correction N(r) on a 3D active box of extents n3 = (nx, ny, nz).
    Returns (hidden 8 x N, y)."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
    assert w.size == NET_WEIGHTS
    n = (ctypes.c_long * 3)(*n3)
    hid = np.empty(8 * r.size)
    y = np.empty(r.size)
    assert _load().og_conv_net_forward(n, _dp(w), _dp(r), _dp(hid), _dp(y)) == 0
    return hid, y


def conv_net_backward(n3, w, r, hid, gy):
    """Weight gradient (and input gradient) of a scalar loss with dLoss/dy = gy."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
    hid = np.ascontiguousarray(hid, dtype=np.float64).reshape(-1)
    gy = np.ascontiguousarray(gy, dtype=np.float64).reshape(-1)
    n = (ctypes.c_long * 3)(*n3)
    gw = np.empty(NET_WEIGHTS)
    dr = np.empty(r.size)
    assert _load().og_conv_net_backward(n, _dp(w), _dp(r), _dp(hid), _dp(gy), _dp(gw),
                                        _dp(dr)) == 0
    return gw, dr


def smoother_loss(g: Grid, a, w, r):
    """Training loss of the learned smoother on one residual sample:
    0.5 ||r - M N(r)||^2, the residual left after one learned correction
    (a local approximate inverse in the residual norm).  Returns (loss, grad)."""
    hid, y = conv_net_forward(g.n, w, r)
    e = np.asarray(r, dtype=np.float64).reshape(-1) - apply_M(g, a, y)
    loss = 0.5 * float(np.dot(e, e))
    gy = -apply_M(g, a, e)           # M is symmetric
    gw, _ = conv_net_backward(g.n, w, r, hid, gy)
    return loss, gw


# ----------------------------------------------------------------------------
# eigen-solvers driving S (Algorithm EigenWave; Arnoldi section)
# ----------------------------------------------------------------------------

def power_iteration(matvec, v0, iters, tol=0.0):
    """Algorithm EigenWave (power iteration on S): v <- S v, beta = (v_new, v_old),
    normalise, stop when ||v_new - sign(beta) v_old|| < tol.  L2 norms are the
    unweighted Euclidean ones over active points.  Returns (v, beta history)."""
    v = np.asarray(v0, dtype=np.float64).reshape(-1)
    v = v / np.linalg.norm(v)
    betas = []
    for _ in range(iters):
        w = matvec(v)
        beta = float(np.dot(w, v))
        w = w / np.linalg.norm(w)
        betas.append(beta)
        done = np.linalg.norm(w - math.copysign(1.0, beta) * v) < tol
        v = w
        if done:
            break
    return v, betas


def _cgs2(V, w):
    """Classical Gram-Schmidt applied twice: returns (w_perp, coefficients)."""
    h1 = V.T @ w
    w = w - V @ h1
    h2 = V.T @ w
    w = w - V @ h2
    return w, h1 + h2


def krylov_schur_eigs(matvec, v0, n_wanted, krylov_dim, tol=1e-10, max_matvecs=2000):
    """Block Arnoldi with thick (Krylov-Schur) restarts for the symmetric S.

    Arnoldi section: Algorithm arnoldi builds S V_m = V_m H_m + F E_m^T with
    Gram-Schmidt (here classical Gram-Schmidt applied twice, and the
    ``h_{j+1,j}`` entry that the listing misprints); the restart keeps the
    wanted Ritz vectors, as IRAM (Algorithm IRAM) and Krylov-Schur do.  The
    wanted set is the ``n_wanted`` largest algebraic Ritz values of S (reading:
    the peak of the filter, not the largest magnitude, holds the eigenvalues
    nearest omega).  ``v0`` is N x b (block size b).  A Ritz pair (theta, x)
    has converged when ||S x - theta x|| <= tol.  Returns (theta, X, matvecs)
    for the converged wanted pairs, by descending theta.  As an iteration path
    this is parity unpinned; its results are pinned by closed-form eigenvalues
    in the tests."""
    V = np.asarray(v0, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    N, b = V.shape
    V, _ = np.linalg.qr(V)
    H = np.zeros((b, 0))       # S V[:, :m] = V[:, :m+b] H   (Krylov-Schur relation)
    m = 0
    nmv = 0
    while True:
        while m < krylov_dim:
            W = np.column_stack([matvec(V[:, m + j]) for j in range(b)])
            nmv += b
            Vk = V[:, :m + b]
            coef = Vk.T @ W
            W = W - Vk @ coef
            coef2 = Vk.T @ W
            W = W - Vk @ coef2
            Q, R = np.linalg.qr(W)
            Hn = np.zeros((m + 2 * b, m + b))
            Hn[:m + b, :m] = H
            Hn[:m + b, m:m + b] = coef + coef2
            Hn[m + b:, m:m + b] = R
            H = Hn
            V = np.column_stack([V, Q])
            m += b
        Hm = 0.5 * (H[:m, :m] + H[:m, :m].T)
        theta, Y = np.linalg.eigh(Hm)
        order = np.argsort(-theta)
        theta, Y = theta[order], Y[:, order]
        coupling = H[m:m + b, :m] @ Y           # b x m
        resid = np.linalg.norm(coupling, axis=0)
        conv = resid[:n_wanted] <= tol
        if conv.all() or nmv >= max_matvecs:
            sel = np.nonzero(conv)[0]
            return theta[sel], V[:, :m] @ Y[:, sel], nmv
        k = min(n_wanted + (m - n_wanted) // 2, m - b)
        X = V[:, :m] @ Y[:, :k]
        Hn = np.zeros((k + b, k))
        Hn[:k, :k] = np.diag(theta[:k])
        Hn[k:, :k] = coupling[:, :k]
        H = Hn
        V = np.column_stack([X, V[:, m:m + b]])
        m = k
