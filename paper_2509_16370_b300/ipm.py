"""Thin ctypes binding of include/rlqr_ipm.h: the batched regularized
interior-point method on the cart with a double pendulum.

Argument marshalling only: the iterations run in the CUDA kernels of
librlqr.so (linearization, the batched LQR solves, the inertia correction and
the line search).  Tensors are torch CUDA tensors; the functions keep the C
names.
"""
from __future__ import annotations

import ctypes

import torch

from . import inputs
from .rlqr import RLQR_FP64, RLQR_MIXED, _check, _ptr, _stream, lib

RLQR_IPM_HESS_EXACT_FP64, RLQR_IPM_HESS_EXACT_FP32, RLQR_IPM_HESS_GAUSS_NEWTON = 0, 1, 2
RUNNING, CONVERGED, ITERATION_LIMIT, RHO_LIMIT = 0, 1, 2, 3
EXPORTED = ("rlqr_ipm_workspace_bytes", "rlqr_ipm_init", "rlqr_ipm_linearize",
            "rlqr_ipm_iterate", "rlqr_ipm_solve", "rlqr_ipm_lqr_view")

_dp = ctypes.c_void_p
_d = ctypes.c_double
_i = ctypes.c_int32


class rlqr_cdp_model(ctypes.Structure):
    _fields_ = [("N", _i), ("dt", _d), ("m0", _d), ("m1", _d), ("m2", _d), ("l1", _d),
                ("l2", _d), ("grav", _d), ("u_max", _d), ("p_max", _d), ("wx", _d * 6),
                ("wu", _d), ("wf", _d * 6)]


class rlqr_ipm_opts(ctypes.Structure):
    _fields_ = [("max_iter", _i), ("tol", _d), ("eta", _d), ("mu0", _d), ("mu_min", _d),
                ("kappa_mu", _d), ("tau", _d), ("armijo", _d), ("ls_steps", _i),
                ("rho_first", _d), ("rho_grow", _d), ("rho_shrink", _d), ("rho_min", _d),
                ("rho_max", _d), ("kappa_sigma", _d), ("s_min", _d), ("hessian", _i),
                ("lqr_prec", _i), ("lqr_max_refine", _i), ("lqr_tol", _d)]


class rlqr_ipm_state(ctypes.Structure):
    _fields_ = [(k, _dp) for k in ("X", "U", "Y", "S", "Z", "mu", "rho", "kkt", "iters",
                                   "factorizations", "status")]


class rlqr_ipm_lqr(ctypes.Structure):
    _fields_ = [(k, _dp) for k in ("Q", "M", "R", "q", "r", "A", "B", "c", "dx", "du", "dy",
                                   "pivot_pd")]


_P = ctypes.POINTER
lib.rlqr_ipm_workspace_bytes.restype = ctypes.c_size_t
lib.rlqr_ipm_workspace_bytes.argtypes = [_i, _P(rlqr_cdp_model), _P(rlqr_ipm_opts)]
lib.rlqr_ipm_init.restype = ctypes.c_int
lib.rlqr_ipm_init.argtypes = [_i, _P(rlqr_cdp_model), _P(rlqr_ipm_opts), _dp, _dp, _dp,
                              _P(rlqr_ipm_state), _dp]
lib.rlqr_ipm_linearize.restype = ctypes.c_int
lib.rlqr_ipm_linearize.argtypes = [_i, _P(rlqr_cdp_model), _P(rlqr_ipm_opts), _dp, _dp,
                                   _P(rlqr_ipm_state), _dp, ctypes.c_size_t, _dp]
lib.rlqr_ipm_iterate.restype = ctypes.c_int
lib.rlqr_ipm_iterate.argtypes = [_i, _P(rlqr_cdp_model), _P(rlqr_ipm_opts), _dp, _dp,
                                 _P(rlqr_ipm_state), _dp, ctypes.c_size_t, _P(_i), _dp]
lib.rlqr_ipm_solve.restype = ctypes.c_int
lib.rlqr_ipm_solve.argtypes = [_i, _P(rlqr_cdp_model), _P(rlqr_ipm_opts), _dp, _dp,
                               _P(rlqr_ipm_state), _dp, ctypes.c_size_t, _P(_i), _dp]
lib.rlqr_ipm_lqr_view.restype = ctypes.c_int
lib.rlqr_ipm_lqr_view.argtypes = [_i, _P(rlqr_cdp_model), _P(rlqr_ipm_opts), _dp,
                                  _P(rlqr_ipm_lqr)]


def make_model(**kw) -> rlqr_cdp_model:
    """The workload's problem data (inputs.CDP_MODEL), with overrides."""
    d = dict(inputs.CDP_MODEL)
    d.update(kw)
    m = rlqr_cdp_model()
    for k, v in d.items():
        if k in ("wx", "wf"):
            getattr(m, k)[:] = [float(t) for t in v]
        else:
            setattr(m, k, v)
    return m


def make_ipm_opts(hessian=RLQR_IPM_HESS_EXACT_FP32, lqr_prec=RLQR_MIXED, **kw) -> rlqr_ipm_opts:
    """The method's constants (the oracle's defaults), with overrides."""
    d = dict(max_iter=300, tol=1e-6, eta=1e3, mu0=0.1, mu_min=1e-8, kappa_mu=10.0, tau=0.995,
             armijo=1e-4, ls_steps=12, rho_first=1e-4, rho_grow=8.0, rho_shrink=3.0,
             rho_min=1e-8, rho_max=1e8, kappa_sigma=1e10, s_min=1e-2, hessian=hessian,
             lqr_prec=lqr_prec, lqr_max_refine=2, lqr_tol=1e-9)
    d.update(kw)
    o = rlqr_ipm_opts()
    for k, v in d.items():
        setattr(o, k, v)
    return o


class IpmState:
    """Device arrays of the iterates and per-instance counters."""

    def __init__(self, count: int, N: int, device="cuda"):
        f = dict(dtype=torch.float64, device=device)
        i = dict(dtype=torch.int32, device=device)
        self.count, self.N = count, N
        self.X = torch.zeros(count, N + 1, 6, **f)
        self.U = torch.zeros(count, N, **f)
        self.Y = torch.zeros(count, N + 1, 6, **f)
        self.S = torch.ones(count, N + 1, 4, **f)
        self.Z = torch.zeros(count, N + 1, 4, **f)
        self.mu = torch.zeros(count, **f)
        self.rho = torch.zeros(count, **f)
        self.kkt = torch.zeros(count, **f)
        self.iters = torch.zeros(count, **i)
        self.factorizations = torch.zeros(count, **i)
        self.status = torch.zeros(count, **i)

    def c_struct(self) -> rlqr_ipm_state:
        return rlqr_ipm_state(*[_ptr(getattr(self, k)) for k, _ in rlqr_ipm_state._fields_])


def rlqr_ipm_workspace_bytes(count: int, model: rlqr_cdp_model, opts: rlqr_ipm_opts) -> int:
    return int(lib.rlqr_ipm_workspace_bytes(count, ctypes.byref(model), ctypes.byref(opts)))


def alloc_ipm_workspace(count: int, model, opts, device="cuda") -> torch.Tensor:
    nb = rlqr_ipm_workspace_bytes(count, model, opts)
    if nb == 0:
        raise ValueError("invalid IPM arguments")
    return torch.empty(nb + 256, dtype=torch.uint8, device=device)


def _aligned(ws: torch.Tensor):
    base = ws.data_ptr()
    off = (-base) % 256
    return ctypes.c_void_p(base + off), ws.numel() - off


def rlqr_ipm_init(model, opts, x0, state: IpmState, U0=None, X0=None, stream=None):
    st = state.c_struct()
    _check(lib.rlqr_ipm_init(state.count, ctypes.byref(model), ctypes.byref(opts), _ptr(x0),
                             _ptr(U0), _ptr(X0), ctypes.byref(st), _stream(stream)),
           "rlqr_ipm_init")


def rlqr_ipm_linearize(model, opts, x0, xg, state: IpmState, ws, stream=None):
    st = state.c_struct()
    p, nb = _aligned(ws)
    _check(lib.rlqr_ipm_linearize(state.count, ctypes.byref(model), ctypes.byref(opts),
                                  _ptr(x0), _ptr(xg), ctypes.byref(st), p, nb, _stream(stream)),
           "rlqr_ipm_linearize")


def rlqr_ipm_iterate(model, opts, x0, xg, state: IpmState, ws, stream=None) -> int:
    st = state.c_struct()
    p, nb = _aligned(ws)
    n = _i(0)
    _check(lib.rlqr_ipm_iterate(state.count, ctypes.byref(model), ctypes.byref(opts), _ptr(x0),
                                _ptr(xg), ctypes.byref(st), p, nb, ctypes.byref(n),
                                _stream(stream)), "rlqr_ipm_iterate")
    return int(n.value)


def rlqr_ipm_solve(model, opts, x0, xg, state: IpmState, ws, stream=None) -> int:
    st = state.c_struct()
    p, nb = _aligned(ws)
    n = _i(0)
    _check(lib.rlqr_ipm_solve(state.count, ctypes.byref(model), ctypes.byref(opts), _ptr(x0),
                              _ptr(xg), ctypes.byref(st), p, nb, ctypes.byref(n),
                              _stream(stream)), "rlqr_ipm_solve")
    return int(n.value)


def rlqr_ipm_lqr_view(model, opts, state: IpmState, ws) -> dict:
    """Torch views of the LQR data of the last Newton system in the workspace
    (instance-major: Q (count, N+1, 6, 6), M (count, N, 6, 1), ...)."""
    out = rlqr_ipm_lqr()
    p, _ = _aligned(ws)
    _check(lib.rlqr_ipm_lqr_view(state.count, ctypes.byref(model), ctypes.byref(opts), p,
                                 ctypes.byref(out)), "rlqr_ipm_lqr_view")
    C, N = state.count, state.N
    shapes = dict(Q=(C, N + 1, 6, 6), M=(C, N, 6, 1), R=(C, N, 1, 1), q=(C, N + 1, 6),
                  r=(C, N, 1), A=(C, N, 6, 6), B=(C, N, 6, 1), c=(C, N + 1, 6),
                  dx=(C, N + 1, 6), du=(C, N, 1), dy=(C, N + 1, 6))
    base = ws.data_ptr()
    views = {}
    for k, shp in shapes.items():
        off = getattr(out, k) - base
        n = 1
        for d in shp:
            n *= d
        views[k] = ws[off:off + 8 * n].view(torch.float64).view(*shp)
    off = out.pivot_pd - base
    views["pivot_pd"] = ws[off:off + C * (N + 1)].view(C, N + 1)
    return views


__all__ = ["RLQR_FP64", "RLQR_MIXED", "make_model", "make_ipm_opts", "IpmState",
           "alloc_ipm_workspace"] + list(EXPORTED)
