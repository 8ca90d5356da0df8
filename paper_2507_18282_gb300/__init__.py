"""GB300 (sm_103a) EigenWave filter-operator library: Python binding.

The functions below carry the names of the C ABI entry points in
include/ew.h and only marshal arguments: every step of the filter operator
runs in the CUDA kernels of libew.so.  Device memory and streams come from
PyTorch (CUDA tensors, torch's current stream).

    g = ew_grid_create(2, (2047, 3071), (1.0, 1.5), order=4, prec="fp32")
    p = filter_params(omega=150.0, num_periods=1)
    ew_filter_apply(g, p, v_in, v_out)          # v_out = S v_in on the GPU
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (EW_BC_DIRICHLET, EW_BC_NEUMANN, EW_EXPLICIT, EW_FP32, EW_FP32X2, EW_FP64, EW_IMPLICIT, EWError, check, lib,
                   ew_filter_info, ew_filter_params, ew_mg_params)

__all__ = ["Grid", "EWError", "ew_grid_create", "ew_grid_create_mapped", "ew_grid_destroy", "filter_params", "mg_params",
           "ew_filter_setup", "ew_choose_num_periods", "ew_filter_apply", "ew_apply_L", "ew_rayleigh",
           "ew_power_iteration",
           "ew_last_error", "LIB_PATH"]

LIB_PATH = _lib.LIB_PATH


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t, dtype, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if t.dtype != dtype:
        raise TypeError("expected dtype %s, got %s" % (dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError("tensor holds %d elements, need %d" % (t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


class Grid:
    """Owner of an ew_grid* handle (ew_grid_create / ew_grid_destroy).

    ``n_interior`` are the interior points per axis, ``bc`` the six face kinds
    (EW_BC_DIRICHLET / EW_BC_NEUMANN), ``n`` the active points per axis (a
    Neumann face's wall points are active) and ``size`` their product."""

    def __init__(self, handle, dim, n_interior, length, order, prec, bc):
        self.handle = handle
        self.dim, self.length, self.order, self.prec = dim, tuple(length), order, prec
        self.n_interior = tuple(n_interior)
        self.bc = tuple(bc)
        self.n = tuple(m + int(bc[2 * a] == EW_BC_NEUMANN) + int(bc[2 * a + 1] == EW_BC_NEUMANN)
                       for a, m in enumerate(self.n_interior))
        self.size = int(np.prod(self.n))

    @property
    def dtype(self):
        import torch
        return torch.float32 if self.prec == EW_FP32 else torch.float64

    def close(self):
        if self.handle:
            lib.ew_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ew_grid_create(dim, n, length, order=2, prec="fp32", bc=None):
    """``n``: interior points per axis; ``bc``: None (all Dirichlet) or 2 dim face
    kinds (-x, +x, -y, +y[, -z, +z]), each "D" / "N" or EW_BC_DIRICHLET / EW_BC_NEUMANN."""
    p = {"fp32": EW_FP32, "fp64": EW_FP64, "fp32x2": EW_FP32X2, EW_FP32: EW_FP32, EW_FP64: EW_FP64,
         EW_FP32X2: EW_FP32X2}[prec]
    kinds = {"D": EW_BC_DIRICHLET, "N": EW_BC_NEUMANN, EW_BC_DIRICHLET: EW_BC_DIRICHLET,
             EW_BC_NEUMANN: EW_BC_NEUMANN}
    faces = [EW_BC_DIRICHLET] * 6
    if bc is not None:
        if len(bc) != 2 * dim:
            raise ValueError("bc needs %d face kinds" % (2 * dim))
        faces[:2 * dim] = [kinds.get(f, f) for f in bc]
    n3 = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    l3 = (ctypes.c_double * 3)(*(list(length) + [1.0] * (3 - len(length))))
    b6 = (ctypes.c_int * 6)(*faces)
    h = ctypes.c_void_p()
    check(lib.ew_grid_create(int(dim), n3, l3, int(order), b6, p, ctypes.byref(h)))
    return Grid(h, dim, n[:dim], length[:dim], order, p, faces[:2 * dim])


def ew_grid_create_mapped(n, xy, prec="fp32"):
    """A curvilinear grid of the unit square's map x = G(r): ``n`` = (n1, n2)
    interior vertices, ``xy`` = vertex coordinates, shape (n2 + 2, n1 + 2, 2)
    (r1 index fastest, boundary vertices included)."""
    p = {"fp32": EW_FP32, "fp64": EW_FP64, EW_FP32: EW_FP32, EW_FP64: EW_FP64}[prec]
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    if xy.shape != (int(n[1]) + 2, int(n[0]) + 2, 2):
        raise ValueError("xy must have shape (n2 + 2, n1 + 2, 2)")
    n2_ = (ctypes.c_int64 * 2)(int(n[0]), int(n[1]))
    h = ctypes.c_void_p()
    check(lib.ew_grid_create_mapped(n2_, xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p, ctypes.byref(h)))
    g = Grid(h, 2, (int(n[0]), int(n[1])), (1.0, 1.0), 2, p, [EW_BC_DIRICHLET] * 4)
    g.mapped = True
    return g


def ew_grid_destroy(grid: Grid):
    grid.close()


def mg_params(pre=2, post=2, max_cycles=1, rtol=0.0, jacobi_weight=0.8, learned_levels=0, weights=None,
              red_black=False, guess="rhs"):
    """guess: "rhs" (0) or "previous" (1), the implicit wave-solve's initial guess."""
    wp = None
    if weights is not None:
        import torch
        wp = _ptr(weights, torch.float32, 432 * max(int(learned_levels), 1))
    gs = {"rhs": 0, "previous": 1}.get(guess, guess)
    m = ew_mg_params(pre, post, max_cycles, rtol, jacobi_weight, learned_levels, wp, int(bool(red_black)), int(gs))
    m._keep = weights
    return m


def filter_params(omega, num_periods=1, steps_per_period=0, cfl=0.8, scheme="explicit",
                  adjust_omega=False, temporal_block=0, mg=None):
    s = {"explicit": EW_EXPLICIT, "implicit": EW_IMPLICIT, EW_EXPLICIT: EW_EXPLICIT,
         EW_IMPLICIT: EW_IMPLICIT}[scheme]
    p = ew_filter_params(float(omega), int(num_periods), int(steps_per_period), float(cfl), s,
                         int(bool(adjust_omega)), int(temporal_block),
                         ctypes.pointer(mg) if mg is not None else None)
    p._keep = mg
    return p


def ew_filter_setup(grid: Grid, params):
    """(info dict, weights c_n as float64 numpy array) of one wave-solve."""
    info = ew_filter_info()
    check(lib.ew_filter_setup(grid.handle, ctypes.byref(params), ctypes.byref(info), None, 0))
    w = np.empty(info.num_steps + 1, dtype=np.float64)
    check(lib.ew_filter_setup(grid.handle, ctypes.byref(params), None,
                              w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), w.size))
    return dict(omega=info.omega_used, Tf=info.final_time, dt=info.dt, alpha_d=info.alpha_d,
                Nt=info.num_steps, steps_per_period=info.steps_per_period), w


def ew_choose_num_periods(grid: Grid, params, n_wanted, krylov_dim, max_periods=1024):
    """(N_p, CR estimate per candidate N_p = 1, 2, 4, ... as a float64 numpy array)."""
    ncand = int(max_periods).bit_length()
    cr = np.zeros(ncand)
    npc = ctypes.c_int(0)
    check(lib.ew_choose_num_periods(grid.handle, ctypes.byref(params), int(n_wanted), int(krylov_dim),
                                    int(max_periods), ctypes.byref(npc),
                                    cr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return npc.value, cr


def ew_filter_apply(grid: Grid, params, v_in, v_out, nvec=None, stream=None):
    nvec = nvec if nvec is not None else max(1, v_in.numel() // grid.size)
    a = _ptr(v_in, grid.dtype, nvec * grid.size)
    b = _ptr(v_out, grid.dtype, nvec * grid.size)
    check(lib.ew_filter_apply(grid.handle, ctypes.byref(params), a, b, int(nvec), _stream(stream)))
    return v_out


def _host_ptr(t, dtype, numel):
    """Data pointer of a contiguous CPU torch tensor (pinned for overlapped copies)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("expected a CPU (host) torch tensor")
    if t.dtype != dtype:
        raise TypeError("expected dtype %s, got %s" % (dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if t.numel() < numel:
        raise ValueError("tensor holds %d elements, need %d" % (t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def ew_filter_apply_host(grid: Grid, params, h_in, h_out, nvec=None, chunk=0, stream=None):
    """v_out = S v_in for vectors in host memory (CPU tensors, ideally pinned),
    copies overlapped with the wave-solves; stream-ordered: synchronise the
    stream before reading h_out."""
    nvec = nvec if nvec is not None else max(1, h_in.numel() // grid.size)
    a = _host_ptr(h_in, grid.dtype, nvec * grid.size)
    b = _host_ptr(h_out, grid.dtype, nvec * grid.size)
    check(lib.ew_filter_apply_host(grid.handle, ctypes.byref(params), a, b, int(nvec), int(chunk), _stream(stream)))
    return h_out


def ew_filter_apply_batched(grids, params, v_in, v_out, nvec=None, stream=None):
    """v_out[q] = S_q v_in[q] for every problem q in one graph-captured launch sequence."""
    n = len(grids)
    G = (ctypes.c_void_p * n)(*[g.handle.value if hasattr(g.handle, "value") else g.handle for g in grids])
    P = (ew_filter_params * n)(*params)
    nvec = list(nvec) if nvec is not None else [1] * n
    if len(nvec) != n:
        raise ValueError("nvec needs one entry per problem")
    vi = (ctypes.c_void_p * n)(*[_ptr(v_in[q], grids[q].dtype, nvec[q] * grids[q].size).value for q in range(n)])
    vo = (ctypes.c_void_p * n)(*[_ptr(v_out[q], grids[q].dtype, nvec[q] * grids[q].size).value for q in range(n)])
    nv = (ctypes.c_int * n)(*[int(k) for k in nvec])
    check(lib.ew_filter_apply_batched(n, G, P, vi, vo, nv, _stream(stream)))
    return v_out


def ew_apply_L(grid: Grid, u, Lu, nvec=None, stream=None):
    nvec = nvec if nvec is not None else max(1, u.numel() // grid.size)
    check(lib.ew_apply_L(grid.handle, _ptr(u, grid.dtype, nvec * grid.size),
                         _ptr(Lu, grid.dtype, nvec * grid.size), int(nvec), _stream(stream)))
    return Lu


def ew_rayleigh(grid: Grid, phi, nvec=None, stream=None):
    """(lambda, eig-res) per vector, as float64 numpy arrays."""
    nvec = nvec if nvec is not None else max(1, phi.numel() // grid.size)
    lam = np.zeros(nvec)
    res = np.zeros(nvec)
    dp = ctypes.POINTER(ctypes.c_double)
    check(lib.ew_rayleigh(grid.handle, _ptr(phi, grid.dtype, nvec * grid.size), int(nvec),
                          lam.ctypes.data_as(dp), res.ctypes.data_as(dp), _stream(stream)))
    return lam, res


def ew_power_iteration(grid: Grid, params, v, iters, tol=0.0, stream=None):
    """Algorithm EigenWave on the GPU.  v is updated in place; returns
    (betas, iterations done, lambda)."""
    betas = np.zeros(max(iters, 1))
    done = ctypes.c_int(0)
    lam = ctypes.c_double(0.0)
    check(lib.ew_power_iteration(grid.handle, ctypes.byref(params), _ptr(v, grid.dtype, grid.size),
                                 int(iters), float(tol),
                                 betas.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.byref(done), ctypes.byref(lam), _stream(stream)))
    return betas[:done.value], done.value, lam.value


def eigs_params(n_wanted, krylov_dim=0, block=1, tol=0.0, max_wave_solves=0, seed=0, refine_fp64=False,
                refine_tol=0.0, lock=False):
    return _lib.ew_eigs_params(int(n_wanted), int(krylov_dim), int(block), float(tol), int(max_wave_solves),
                               int(seed), int(refine_fp64), float(refine_tol), int(bool(lock)))


def ew_arnoldi_eigs(grid: Grid, params, eigs, start=None, vecs=None, stream=None, allow_noconv=False):
    """Block Krylov-Schur on S.  Returns (lambda (n_wanted,), report dict, status).
    `start` (FP64 CUDA tensor, N x block column-major) and `vecs` (FP64 CUDA
    tensor receiving N x n_wanted eigenvectors) are optional."""
    nw = eigs.n_wanted
    lam = np.zeros(nw)
    rep = _lib.ew_eigs_report()
    import torch
    sp = _ptr(start, torch.float64, grid.size * max(eigs.block, 1)) if start is not None else None
    vp = _ptr(vecs, torch.float64, grid.size * nw) if vecs is not None else None
    st = lib.ew_arnoldi_eigs(grid.handle, ctypes.byref(params), ctypes.byref(eigs), sp,
                             lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), vp, ctypes.byref(rep),
                             _stream(stream))
    if st != _lib.EW_OK and not (allow_noconv and st == _lib.EW_ENOCONV):
        check(st)
    report = dict(n_converged=rep.n_converged, wave_solves=rep.wave_solves,
                  wave_solves_fp64=rep.wave_solves_fp64, restarts=rep.restarts, seconds=rep.seconds,
                  beta=np.array(rep.beta[:nw]), eig_res=np.array(rep.eig_res[:nw]),
                  lambda_stage1=np.array(rep.lambda_stage1[:nw]),
                  eig_res_stage1=np.array(rep.eig_res_stage1[:nw]),
                  lambda_rel_change=np.array(rep.lambda_rel_change[:nw]))
    return lam, report, st


def tb2d_choice(grid: Grid, nvec=1):
    """The tuned 2D blocked-step variant for this grid and nvec: dict(kernel,
    depth, tile) or None if none has been tuned yet."""
    buf = ctypes.create_string_buffer(256)
    b, tx, ty = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    st = lib.ew_tuned_variant(grid.handle, int(nvec), buf, 256, ctypes.byref(b), ctypes.byref(tx), ctypes.byref(ty))
    if st != _lib.EW_OK:
        return None
    return dict(kernel=buf.value.decode(), depth=b.value, tile=[tx.value, ty.value])


def _report_dict(rep, nw):
    return dict(n_converged=rep.n_converged, wave_solves=rep.wave_solves,
                wave_solves_fp64=rep.wave_solves_fp64, restarts=rep.restarts, seconds=rep.seconds,
                beta=np.array(rep.beta[:nw]), eig_res=np.array(rep.eig_res[:nw]),
                lambda_stage1=np.array(rep.lambda_stage1[:nw]),
                eig_res_stage1=np.array(rep.eig_res_stage1[:nw]),
                lambda_rel_change=np.array(rep.lambda_rel_change[:nw]))


def ew_arnoldi_eigs_batched(grids, params, eigs, vecs=None, stream=None, allow_noconv=False):
    """Eigen-solves of len(grids) problems with batched filter applications.
    `params` and `eigs` hold one entry per problem; `vecs` (optional) one FP64
    CUDA tensor (N_q x n_wanted_q) or None per problem.  Returns (list of
    lambda arrays, list of report dicts, list of statuses, batched rounds)."""
    import torch
    n = len(grids)
    G = (ctypes.c_void_p * n)(*[g.handle.value if hasattr(g.handle, "value") else g.handle for g in grids])
    P = (ew_filter_params * n)(*params)
    E = (_lib.ew_eigs_params * n)(*eigs)
    lams = [np.zeros(e.n_wanted) for e in eigs]
    L = (ctypes.POINTER(ctypes.c_double) * n)(*[x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for x in lams])
    V = None
    if vecs is not None:
        V = (ctypes.c_void_p * n)(*[(_ptr(vecs[q], torch.float64, grids[q].size * eigs[q].n_wanted).value
                                     if vecs[q] is not None else None) for q in range(n)])
    R = (_lib.ew_eigs_report * n)()
    S = (ctypes.c_int * n)()
    rounds = ctypes.c_int(0)
    st = lib.ew_arnoldi_eigs_batched(n, G, P, E, L, V, R, S, ctypes.byref(rounds), _stream(stream))
    if st != _lib.EW_OK and not (allow_noconv and all(x in (_lib.EW_OK, _lib.EW_ENOCONV) for x in S)):
        check(st)
    return lams, [_report_dict(R[q], eigs[q].n_wanted) for q in range(n)], list(S), rounds.value


def ew_implicit_step_mg(grid: Grid, half_dt2, rhs, x, mg, stream=None):
    """Multigrid solve of (I - half_dt2 L_h) x = rhs; x holds the initial guess
    and receives the result.  Returns (convergence factor, cycles run)."""
    conv = ctypes.c_double(0.0)
    cyc = ctypes.c_int(0)
    check(lib.ew_implicit_step_mg(grid.handle, float(half_dt2), _ptr(rhs, grid.dtype, grid.size),
                                  _ptr(x, grid.dtype, grid.size), ctypes.byref(mg), ctypes.byref(conv),
                                  ctypes.byref(cyc), _stream(stream)))
    return conv.value, cyc.value


def ew_smoother_forward(grid: Grid, weights, r, y, stream=None):
    import torch
    check(lib.ew_smoother_forward(grid.handle, _ptr(weights, torch.float32, 432), _ptr(r, grid.dtype, grid.size),
                                  _ptr(y, grid.dtype, grid.size), _stream(stream)))
    return y


def ew_smoother_backward(grid: Grid, weights, r, gy, grad, stream=None):
    import torch
    check(lib.ew_smoother_backward(grid.handle, _ptr(weights, torch.float32, 432), _ptr(r, grid.dtype, grid.size),
                                   _ptr(gy, grid.dtype, grid.size), _ptr(grad, torch.float32, 432),
                                   _stream(stream)))
    return grad


def ew_smoother_train(grid: Grid, half_dt2, weights, steps=200, samples=6, lr=1e-3, pre=2, post=2,
                      jacobi_weight=0.8, seed=1, accept_cycles=6, stream=None):
    """Train the learned smoother in place (weights: 432 FP32 CUDA tensor).
    Returns the report as a dict."""
    import torch
    tp = _lib.ew_train_params(int(steps), int(samples), float(lr), int(pre), int(post), float(jacobi_weight),
                              int(seed), int(accept_cycles))
    rep = _lib.ew_train_report()
    check(lib.ew_smoother_train(grid.handle, float(half_dt2), ctypes.byref(tp), _ptr(weights, torch.float32, 432),
                                ctypes.byref(rep), _stream(stream)))
    return dict(loss_first=rep.loss_first, loss_last=rep.loss_last, conv_plain=rep.conv_plain,
                conv_learned=rep.conv_learned, accepted=bool(rep.accepted))


def ew_profile_enable(on=True):
    check(lib.ew_profile_enable(int(bool(on))))


def ew_profile_read():
    """Totals since the last read: launches, fused_launches, fused_ms, fused_cell_steps, fused_points,
    mg_cycles, mg_solves."""
    p = _lib.ew_profile()
    check(lib.ew_profile_read(ctypes.byref(p)))
    return dict(launches=p.launches, fused_launches=p.fused_launches, fused_ms=p.fused_ms,
                fused_cell_steps=p.fused_cell_steps, fused_points=p.fused_points, mg_cycles=p.mg_cycles,
                mg_solves=p.mg_solves)


def ew_last_error() -> str:
    return _lib.last_error()
