"""Thin Python binding of the C ABI in include/rlqr.h (ctypes).

Argument marshalling only: every step of the solve runs in the CUDA kernels of
librlqr.so.  PyTorch provides device memory and streams.  The functions keep
the C names (rlqr_factor, rlqr_solve, rlqr_residual, rlqr_solve_batched, ...)
and take torch tensors where the C ABI takes device pointers.

The library is loaded from paper_2509_16370_b300/_lib/librlqr.so; if it is
missing this module raises at import time (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librlqr.so")

RLQR_OK, RLQR_NOT_PD, RLQR_ERR_ARG, RLQR_ERR_SINGULAR = 0, 1, 2, 3
RLQR_ERR_NOT_CONVERGED, RLQR_ERR_TIMEOUT, RLQR_ERR_WORKSPACE, RLQR_ERR_CUDA = 4, 5, 6, 7
RLQR_OPT_SYNC = 1
RLQR_ALGO_AUTO, RLQR_ALGO_SEQ, RLQR_ALGO_SCAN = 0, 1, 2
RLQR_FP64, RLQR_MIXED = 0, 1

EXPORTED = ("rlqr_default_opts", "rlqr_version", "rlqr_status_string", "rlqr_workspace_bytes",
            "rlqr_factor", "rlqr_solve", "rlqr_residual", "rlqr_batched_workspace_bytes",
            "rlqr_solve_batched", "rlqr_instrument", "rlqr_instrument_report",
            "rlqr_solve_noalloc")
NOALLOC_SCRATCH_BYTES = 8 << 20

_dp = ctypes.c_void_p


class rlqr_problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("nx", ctypes.c_int32), ("nu", ctypes.c_int32),
                ("Q", _dp), ("M", _dp), ("R", _dp), ("q", _dp), ("r", _dp), ("A", _dp),
                ("B", _dp), ("c", _dp), ("delta", ctypes.c_double)]


class rlqr_opts(ctypes.Structure):
    _fields_ = [("max_refine", ctypes.c_int32), ("tol", ctypes.c_double), ("algo", ctypes.c_int),
                ("prec", ctypes.c_int), ("flags", ctypes.c_int32)]


class rlqr_batch(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("h_N", _dp), ("h_nx", _dp), ("h_nu", _dp),
                ("N", _dp), ("nx", _dp), ("nu", _dp)] + [
        (f"off_{k}", _dp) for k in ("Q", "M", "R", "q", "r", "A", "B", "c", "x", "u", "y",
                                    "flag")] + [
        ("delta", _dp)] + [(k, _dp) for k in ("Q", "M", "R", "q", "r", "A", "B", "c", "x", "u",
                                              "y", "pivot_pd")]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2509_16370_b300.csrc.build` (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    st, sz = ctypes.c_int, ctypes.c_size_t
    P = ctypes.POINTER
    lib.rlqr_default_opts.restype = rlqr_opts
    lib.rlqr_version.restype = ctypes.c_char_p
    lib.rlqr_status_string.restype = ctypes.c_char_p
    lib.rlqr_status_string.argtypes = [st]
    lib.rlqr_workspace_bytes.restype = sz
    lib.rlqr_workspace_bytes.argtypes = [ctypes.c_int32] * 3 + [P(rlqr_opts)]
    lib.rlqr_factor.restype = st
    lib.rlqr_factor.argtypes = [P(rlqr_problem), P(rlqr_opts), _dp, sz, _dp, _dp, _dp]
    lib.rlqr_solve.restype = st
    lib.rlqr_solve.argtypes = [P(rlqr_problem), P(rlqr_opts), _dp, sz, _dp, _dp, _dp, _dp, _dp,
                               _dp, _dp]
    lib.rlqr_residual.restype = st
    lib.rlqr_residual.argtypes = [P(rlqr_problem), _dp, _dp, _dp, _dp, _dp, _dp]
    lib.rlqr_batched_workspace_bytes.restype = sz
    lib.rlqr_batched_workspace_bytes.argtypes = [P(rlqr_batch), P(rlqr_opts)]
    lib.rlqr_solve_batched.restype = st
    lib.rlqr_solve_batched.argtypes = [P(rlqr_batch), P(rlqr_opts), _dp, sz, _dp, _dp, _dp, _dp]
    lib.rlqr_solve_noalloc.restype = st
    lib.rlqr_solve_noalloc.argtypes = [P(rlqr_problem), P(rlqr_opts), _dp, _dp, _dp, _dp, _dp, _dp,
                                       _dp]
    i32, dbl = ctypes.c_int32, ctypes.c_double
    for name, args in (
            ("rlqr_shard_element", [P(rlqr_problem), P(rlqr_opts), _dp, sz, _dp, _dp]),
            ("rlqr_shard_boundary", [i32, i32, i32, i32, _dp, _dp, _dp, _dp, _dp]),
            ("rlqr_shard_pmap", [P(rlqr_problem), P(rlqr_opts), _dp, sz, _dp, _dp, _dp]),
            ("rlqr_shard_p_end", [i32, i32, i32, _dp, _dp, _dp, _dp, _dp]),
            ("rlqr_shard_x_offset", [i32, _dp, _dp, _dp, _dp, _dp]),
            ("rlqr_shard_x_start", [i32, i32, _dp, _dp, _dp, _dp]),
            ("rlqr_shard_entry", [i32, dbl, _dp, _dp, _dp, _dp, _dp])):
        getattr(lib, name).restype = st
        getattr(lib, name).argtypes = args
    lib.rlqr_cross_scratch_bytes.restype = sz
    lib.rlqr_cross_scratch_bytes.argtypes = [ctypes.c_int32] * 4 + [P(rlqr_opts)]
    lib.rlqr_solve_cross.restype = st
    lib.rlqr_solve_cross.argtypes = [P(rlqr_problem), P(rlqr_opts), _dp, sz, ctypes.c_int32, _dp,
                                     _dp, _dp, _dp, sz, _dp, _dp, _dp, _dp, _dp, _dp]
    lib.rlqr_autotune_scan.restype = st
    lib.rlqr_autotune_scan.argtypes = [P(rlqr_problem), P(rlqr_opts), _dp, sz, _dp, _dp, _dp, _dp,
                                       P(ctypes.c_int32), P(ctypes.c_double), _dp]
    lib.rlqr_tune_scan_set.restype = st
    lib.rlqr_tune_scan_set.argtypes = [ctypes.c_int32] * 3 + [P(rlqr_opts), ctypes.c_int32]
    lib.rlqr_autotune_batched.restype = st
    lib.rlqr_autotune_batched.argtypes = [P(rlqr_batch), P(rlqr_opts), _dp, sz, _dp,
                                          P(ctypes.c_int32), P(ctypes.c_double), _dp]
    lib.rlqr_tune_batched_set.restype = st
    lib.rlqr_tune_batched_set.argtypes = [P(rlqr_batch), P(rlqr_opts), ctypes.c_int32]
    lib.rlqr_tune_reset.restype = st
    lib.rlqr_tune_reset.argtypes = []
    lib.rlqr_diag_workspace_bytes.restype = sz
    lib.rlqr_diag_workspace_bytes.argtypes = [ctypes.c_int32] * 3 + [P(rlqr_opts)]
    lib.rlqr_solve_diag.restype = st
    lib.rlqr_solve_diag.argtypes = [P(rlqr_problem), _dp, P(rlqr_opts), _dp, sz, _dp, _dp, _dp,
                                    _dp, _dp, _dp, _dp]
    lib.rlqr_measure_pipes_bytes.restype = sz
    lib.rlqr_measure_pipes_bytes.argtypes = []
    lib.rlqr_measure_pipes.restype = st
    lib.rlqr_measure_pipes.argtypes = [_dp, sz] + [P(ctypes.c_double)] * 3
    lib.rlqr_measure_tf32.restype = st
    lib.rlqr_measure_tf32.argtypes = [_dp, sz, P(ctypes.c_double)]
    lib.rlqr_instrument.restype = st
    lib.rlqr_instrument.argtypes = [ctypes.c_int]
    lib.rlqr_instrument_report.restype = ctypes.c_int
    lib.rlqr_instrument_report.argtypes = [ctypes.c_int, P(ctypes.c_char_p),
                                           P(ctypes.c_int64), P(ctypes.c_double)]
    return lib


lib = _load()


class RlqrError(RuntimeError):
    pass


def _check(code: int, what: str):
    if code != RLQR_OK:
        raise RlqrError(f"{what}: {lib.rlqr_status_string(code).decode()} ({code})")


def _check_call(code: int, what: str) -> int:
    """Raise for a failed call (arguments, workspace, CUDA); return an
    instance status (what RLQR_OPT_SYNC calls report) unchanged."""
    if code in (RLQR_ERR_ARG, RLQR_ERR_WORKSPACE, RLQR_ERR_CUDA):
        _check(code, what)
    return int(code)


def _ptr(t):
    if t is None:
        return None
    assert t.is_contiguous(), "tensors passed to librlqr must be contiguous"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def version() -> str:
    return lib.rlqr_version().decode()


def make_opts(prec=RLQR_FP64, algo=RLQR_ALGO_AUTO, tol=1e-9, max_refine=3,
              sync=False) -> rlqr_opts:
    o = lib.rlqr_default_opts()
    o.prec, o.algo, o.tol, o.max_refine = int(prec), int(algo), float(tol), int(max_refine)
    o.flags = RLQR_OPT_SYNC if sync else 0
    return o


def rlqr_instrument(enable: bool):
    _check(lib.rlqr_instrument(1 if enable else 0), "rlqr_instrument")


def rlqr_instrument_report(max_kernels: int = 32) -> dict:
    """{kernel name: (launches, total ms)} of the launches since rlqr_instrument."""
    names = (ctypes.c_char_p * max_kernels)()
    launches = (ctypes.c_int64 * max_kernels)()
    ms = (ctypes.c_double * max_kernels)()
    k = lib.rlqr_instrument_report(max_kernels, names, launches, ms)
    if k < 0:
        raise RlqrError("rlqr_instrument_report: CUDA error")
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(k)}


# ------------------------------------------------------------ single instance

@dataclass
class DeviceProblem:
    """One instance's FP64 arrays on the device (stage-major, contiguous)."""
    N: int
    n: int
    m: int
    Q: torch.Tensor
    M: torch.Tensor
    R: torch.Tensor
    q: torch.Tensor
    r: torch.Tensor
    A: torch.Tensor
    B: torch.Tensor
    c: torch.Tensor
    delta: float

    @staticmethod
    def from_host(p, device="cuda") -> "DeviceProblem":
        t = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k), dtype=np.float64)).to(device)
             for k in ("Q", "M", "R", "q", "r", "A", "B", "c")}
        return DeviceProblem(p.N, p.n, p.m, delta=float(p.delta), **t)

    def c_struct(self) -> rlqr_problem:
        s = rlqr_problem()
        s.N, s.nx, s.nu, s.delta = self.N, self.n, self.m, float(self.delta)
        for k in ("Q", "M", "R", "q", "r", "A", "B", "c"):
            setattr(s, k, _ptr(getattr(self, k)).value)
        return s


def rlqr_workspace_bytes(N: int, nx: int, nu: int, opts: rlqr_opts) -> int:
    return int(lib.rlqr_workspace_bytes(N, nx, nu, ctypes.byref(opts)))


def alloc_workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """Caller-owned workspace (torch allocations are 256-byte aligned)."""
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def rlqr_factor(prob: DeviceProblem, opts: rlqr_opts, ws: torch.Tensor, pivot_pd: torch.Tensor,
                status: torch.Tensor | None = None, stream=None):
    ps = prob.c_struct()
    return _check_call(lib.rlqr_factor(ctypes.byref(ps), ctypes.byref(opts), _ptr(ws), ws.numel(),
                                       _ptr(pivot_pd), _ptr(status), _stream(stream)),
                       "rlqr_factor")


def rlqr_solve(prob: DeviceProblem, opts: rlqr_opts, ws: torch.Tensor, x, u, y, rel_resid=None,
               iters=None, status=None, stream=None):
    ps = prob.c_struct()
    return _check_call(lib.rlqr_solve(ctypes.byref(ps), ctypes.byref(opts), _ptr(ws), ws.numel(),
                                      _ptr(x), _ptr(u), _ptr(y), _ptr(rel_resid), _ptr(iters),
                                      _ptr(status), _stream(stream)), "rlqr_solve")


def rlqr_residual(prob: DeviceProblem, x, u, y, res=None, norms=None, stream=None):
    ps = prob.c_struct()
    _check(lib.rlqr_residual(ctypes.byref(ps), _ptr(x), _ptr(u), _ptr(y), _ptr(res), _ptr(norms),
                             _stream(stream)), "rlqr_residual")


def rlqr_solve_noalloc(prob: DeviceProblem, opts: rlqr_opts, x, u, y, pivot_pd, rel_resid=None,
                       status=None, stream=None):
    """Factor + solve one instance with the library's static scratch instead
    of a workspace: for callers that must not allocate device memory (see
    include/rlqr.h).  Concurrent calls on one device race on that scratch."""
    ps = prob.c_struct()
    return _check_call(lib.rlqr_solve_noalloc(ctypes.byref(ps), ctypes.byref(opts), _ptr(x),
                                              _ptr(u), _ptr(y), _ptr(pivot_pd), _ptr(rel_resid),
                                              _ptr(status), _stream(stream)),
                       "rlqr_solve_noalloc")


# ------------------------------------------------------------------- batches

@dataclass
class DeviceBatch:
    """Pooled device buffers of a batch plus the per-instance offset arrays.

    Works for uniform and ragged batches alike.  Instance b's arrays start at
    element offsets off_*[b] of the pooled buffers."""
    count: int
    h_dims: np.ndarray          # (count, 3) int32 host copy of (N, nx, nu)
    dims: torch.Tensor          # (3, count) int32 device
    offs: dict                  # name -> int64 device tensor [count]
    delta: torch.Tensor         # float64 [count]
    bufs: dict                  # name -> pooled float64 device tensor
    x: torch.Tensor
    u: torch.Tensor
    y: torch.Tensor
    pivot_pd: torch.Tensor
    _h_cols: tuple = ()
    _struct: rlqr_batch | None = None

    @staticmethod
    def from_problems(probs, device="cuda") -> "DeviceBatch":
        dims = np.array([[p.N, p.n, p.m] for p in probs], dtype=np.int32)
        sizes = {
            "Q": [(p.N + 1) * p.n * p.n for p in probs], "M": [p.N * p.n * p.m for p in probs],
            "R": [p.N * p.m * p.m for p in probs], "q": [(p.N + 1) * p.n for p in probs],
            "r": [p.N * p.m for p in probs], "A": [p.N * p.n * p.n for p in probs],
            "B": [p.N * p.n * p.m for p in probs], "c": [(p.N + 1) * p.n for p in probs],
            "x": [(p.N + 1) * p.n for p in probs], "u": [p.N * p.m for p in probs],
            "y": [(p.N + 1) * p.n for p in probs], "flag": [p.N + 1 for p in probs]}
        offs_h = {k: np.concatenate([[0], np.cumsum(v)[:-1]]).astype(np.int64)
                  for k, v in sizes.items()}
        bufs = {}
        for k in ("Q", "M", "R", "q", "r", "A", "B", "c"):
            flat = np.concatenate([np.ascontiguousarray(getattr(p, k), np.float64).ravel()
                                   for p in probs])
            bufs[k] = torch.from_numpy(flat).to(device)
        return DeviceBatch._finish(len(probs), dims, offs_h, sizes, bufs,
                                   np.array([p.delta for p in probs], np.float64), device)

    @staticmethod
    def from_uniform(batch, device="cuda", pinned_host=None) -> "DeviceBatch":
        """A uniform host batch (stacked arrays) without per-instance copies."""
        B, N, n, m = batch.count, batch.N, batch.n, batch.m
        dims = np.tile(np.array([[N, n, m]], np.int32), (B, 1))
        per = {"Q": (N + 1) * n * n, "M": N * n * m, "R": N * m * m, "q": (N + 1) * n,
               "r": N * m, "A": N * n * n, "B": N * n * m, "c": (N + 1) * n, "x": (N + 1) * n,
               "u": N * m, "y": (N + 1) * n, "flag": N + 1}
        offs_h = {k: (np.arange(B, dtype=np.int64) * v) for k, v in per.items()}
        sizes = {k: [v] * B for k, v in per.items()}
        bufs = {k: torch.from_numpy(np.ascontiguousarray(getattr(batch, k), np.float64).reshape(-1))
                .to(device) for k in ("Q", "M", "R", "q", "r", "A", "B", "c")}
        return DeviceBatch._finish(B, dims, offs_h, sizes, bufs,
                                   np.asarray(batch.delta, np.float64), device)

    @staticmethod
    def _finish(count, dims, offs_h, sizes, bufs, delta, device):
        offs = {k: torch.from_numpy(v).to(device) for k, v in offs_h.items()}
        tot = {k: int(sum(v)) for k, v in sizes.items()}
        x = torch.zeros(tot["x"], dtype=torch.float64, device=device)
        u = torch.zeros(tot["u"], dtype=torch.float64, device=device)
        y = torch.zeros(tot["y"], dtype=torch.float64, device=device)
        flags = torch.zeros(tot["flag"], dtype=torch.uint8, device=device)
        hcols = tuple(np.ascontiguousarray(dims[:, i]) for i in range(3))
        db = DeviceBatch(count, dims, torch.from_numpy(np.ascontiguousarray(dims.T)).to(device),
                         offs, torch.from_numpy(delta).to(device), bufs, x, u, y, flags, hcols)
        db._offs_h = offs_h
        return db

    def c_struct(self) -> rlqr_batch:
        s = rlqr_batch()
        s.count = self.count
        s.h_N, s.h_nx, s.h_nu = (c.ctypes.data for c in self._h_cols)
        s.N = self.dims[0].data_ptr()
        s.nx = self.dims[1].data_ptr()
        s.nu = self.dims[2].data_ptr()
        for k, t in self.offs.items():
            setattr(s, f"off_{k}", t.data_ptr())
        s.delta = self.delta.data_ptr()
        for k, t in self.bufs.items():
            setattr(s, k, t.data_ptr())
        s.x, s.u, s.y, s.pivot_pd = (self.x.data_ptr(), self.u.data_ptr(), self.y.data_ptr(),
                                     self.pivot_pd.data_ptr())
        self._struct = s
        return s

    def instance_view(self, b: int):
        """(x, u, y, flags) host arrays of instance b (copies back)."""
        N, n, m = (int(v) for v in self.h_dims[b])
        o = self._offs_h
        x = self.x[o["x"][b]:o["x"][b] + (N + 1) * n].view(N + 1, n).cpu().numpy()
        u = self.u[o["u"][b]:o["u"][b] + N * m].view(N, m).cpu().numpy()
        y = self.y[o["y"][b]:o["y"][b] + (N + 1) * n].view(N + 1, n).cpu().numpy()
        f = self.pivot_pd[o["flag"][b]:o["flag"][b] + N + 1].cpu().numpy()
        return x, u, y, f


def rlqr_batched_workspace_bytes(batch: DeviceBatch, opts: rlqr_opts) -> int:
    s = batch.c_struct()
    return int(lib.rlqr_batched_workspace_bytes(ctypes.byref(s), ctypes.byref(opts)))


def rlqr_solve_batched(batch: DeviceBatch, opts: rlqr_opts, ws: torch.Tensor, status=None,
                       rel_resid=None, iters=None, stream=None):
    s = batch.c_struct()
    _check(lib.rlqr_solve_batched(ctypes.byref(s), ctypes.byref(opts), _ptr(ws), ws.numel(),
                                  _ptr(status), _ptr(rel_resid), _ptr(iters), _stream(stream)),
           "rlqr_solve_batched")


# ------------------------------------------------------------ horizon shards
# Building blocks of the sharded long-horizon solve (see shard.py); every
# tensor is a contiguous FP64 CUDA tensor.

def rlqr_shard_element(shard: "DeviceProblem", opts: rlqr_opts, ws: torch.Tensor, elem, stream=None):
    ps = shard.c_struct()
    _check(lib.rlqr_shard_element(ctypes.byref(ps), ctypes.byref(opts), _ptr(ws), ws.numel(),
                                  _ptr(elem), _stream(stream)), "rlqr_shard_element")


def rlqr_shard_boundary(G: int, g: int, nx: int, nu: int, elems, QN, P_end, P_start=None,
                        stream=None):
    _check(lib.rlqr_shard_boundary(G, g, nx, nu, _ptr(elems), _ptr(QN), _ptr(P_end),
                                   _ptr(P_start), _stream(stream)), "rlqr_shard_boundary")


def rlqr_shard_pmap(shard: "DeviceProblem", opts: rlqr_opts, ws: torch.Tensor, Phi, phi,
                    stream=None):
    ps = shard.c_struct()
    _check(lib.rlqr_shard_pmap(ctypes.byref(ps), ctypes.byref(opts), _ptr(ws), ws.numel(),
                               _ptr(Phi), _ptr(phi), _stream(stream)), "rlqr_shard_pmap")


def rlqr_shard_p_end(G: int, g: int, nx: int, Phis, phis, qN, p_end, stream=None):
    _check(lib.rlqr_shard_p_end(G, g, nx, _ptr(Phis), _ptr(phis), _ptr(qN), _ptr(p_end),
                                _stream(stream)), "rlqr_shard_p_end")


def rlqr_shard_x_offset(nx: int, Phi, x_first, x_last, psi, stream=None):
    _check(lib.rlqr_shard_x_offset(nx, _ptr(Phi), _ptr(x_first), _ptr(x_last), _ptr(psi),
                                   _stream(stream)), "rlqr_shard_x_offset")


def rlqr_shard_x_start(g: int, nx: int, Phis, psis, x_start, stream=None):
    _check(lib.rlqr_shard_x_start(g, nx, _ptr(Phis), _ptr(psis), _ptr(x_start),
                                  _stream(stream)), "rlqr_shard_x_start")


def rlqr_shard_entry(nx: int, delta: float, P_start, x_start, x_first, c0, stream=None):
    _check(lib.rlqr_shard_entry(nx, float(delta), _ptr(P_start), _ptr(x_start), _ptr(x_first),
                                _ptr(c0), _stream(stream)), "rlqr_shard_entry")


def rlqr_measure_pipes() -> dict:
    """Measured FP64 / FP32 / packed-FP32 FMA rates and the TF32 mma.sync
    rate of the current device in TFLOP/s (synchronous microbenchmarks; the
    sink buffer is a torch tensor)."""
    nb = int(lib.rlqr_measure_pipes_bytes())
    buf = torch.empty(max(nb, 8), dtype=torch.uint8, device="cuda")
    v = [ctypes.c_double() for _ in range(3)]
    _check(lib.rlqr_measure_pipes(_ptr(buf), nb, *[ctypes.byref(x) for x in v]),
           "rlqr_measure_pipes")
    t = ctypes.c_double()
    _check(lib.rlqr_measure_tf32(_ptr(buf), nb, ctypes.byref(t)), "rlqr_measure_tf32")
    torch.cuda.synchronize()
    return dict(fp64_tflops=v[0].value, fp32_tflops=v[1].value, fp32x2_tflops=v[2].value,
                tf32_mma_tflops=t.value)


def rlqr_cross_scratch_bytes(N: int, nx: int, nu: int, p: int, opts: rlqr_opts) -> int:
    return int(lib.rlqr_cross_scratch_bytes(N, nx, nu, p, ctypes.byref(opts)))


def rlqr_solve_cross(prob: "DeviceProblem", opts: rlqr_opts, ws: torch.Tensor, J, H, r_theta,
                     scratch: torch.Tensor, x, u, y, dtheta, status=None, stream=None) -> int:
    """Cross-stage variables (include/rlqr.h): J is a (p, L) FP64 tensor of
    columns in the right-hand side's layout, H (p, p), r_theta (p,)."""
    ps = prob.c_struct()
    return _check_call(lib.rlqr_solve_cross(
        ctypes.byref(ps), ctypes.byref(opts), _ptr(ws), ws.numel(), int(J.shape[0]), _ptr(J),
        _ptr(H), _ptr(r_theta), _ptr(scratch), scratch.numel(), _ptr(x), _ptr(u), _ptr(y),
        _ptr(dtheta), _ptr(status), _stream(stream)), "rlqr_solve_cross")



def rlqr_diag_workspace_bytes(N: int, nx: int, nu: int, opts: rlqr_opts) -> int:
    return int(lib.rlqr_diag_workspace_bytes(N, nx, nu, ctypes.byref(opts)))


def rlqr_solve_diag(prob: "DeviceProblem", delta_diag, opts: rlqr_opts, ws: torch.Tensor, x, u, y,
                    pivot_pd, rel_resid=None, status=None, stream=None) -> int:
    """General diagonal Delta_i (delta_diag: device (N+1, nx) FP64)."""
    ps = prob.c_struct()
    return _check_call(lib.rlqr_solve_diag(ctypes.byref(ps), _ptr(delta_diag), ctypes.byref(opts),
                                           _ptr(ws), ws.numel(), _ptr(x), _ptr(u), _ptr(y),
                                           _ptr(pivot_pd), _ptr(rel_resid), _ptr(status),
                                           _stream(stream)), "rlqr_solve_diag")


SCAN_CHUNK_CANDIDATES = (148, 296, 444, 592, 888)


def rlqr_autotune_scan(prob: "DeviceProblem", opts: rlqr_opts, ws: torch.Tensor, x, u, y,
                       pivot_pd, stream=None):
    """Time the scan's chunk counts on `prob` and record the fastest for its
    shape; returns (chunks, ms of one factor + solve)."""
    ps = prob.c_struct()
    c = ctypes.c_int32(0)
    t = ctypes.c_double(0.0)
    _check(lib.rlqr_autotune_scan(ctypes.byref(ps), ctypes.byref(opts), _ptr(ws), ws.numel(),
                                  _ptr(x), _ptr(u), _ptr(y), _ptr(pivot_pd), ctypes.byref(c),
                                  ctypes.byref(t), _stream(stream)), "rlqr_autotune_scan")
    return int(c.value), float(t.value)


def rlqr_tune_scan_set(N: int, nx: int, nu: int, opts: rlqr_opts, chunks: int):
    _check(lib.rlqr_tune_scan_set(N, nx, nu, ctypes.byref(opts), chunks), "rlqr_tune_scan_set")


def rlqr_tune_reset():
    _check(lib.rlqr_tune_reset(), "rlqr_tune_reset")


RES_ROUTE_WARP, RES_ROUTE_GRID, RES_ROUTE_FUSED = 1, 2, 5
# the same residual routes with refinement passes on two warps per instance
RES_ROUTE_WARP_DUO, RES_ROUTE_FUSED_DUO = 6, 7
SWEEP_ROUTE_STREAMS, SWEEP_ROUTE_PERSISTENT = 3, 4


def rlqr_autotune_batched(batch: "DeviceBatch", opts: rlqr_opts, ws: torch.Tensor, status=None,
                          stream=None):
    """Time the routes of the batch -- the residual / refinement routes of a
    uniform batch (1, 2 and, mixed, 5, 6, 7), the sweep routes (class
    streams / persistent launch) of a ragged one -- and record the fastest
    for its shape; returns (route, ms of one rlqr_solve_batched)."""
    bs = batch.c_struct()
    r = ctypes.c_int32(0)
    t = ctypes.c_double(0.0)
    _check(lib.rlqr_autotune_batched(ctypes.byref(bs), ctypes.byref(opts), _ptr(ws), ws.numel(),
                                     _ptr(status), ctypes.byref(r), ctypes.byref(t),
                                     _stream(stream)), "rlqr_autotune_batched")
    return int(r.value), float(t.value)


def rlqr_tune_batched_set(batch: "DeviceBatch", opts: rlqr_opts, route: int):
    bs = batch.c_struct()
    _check(lib.rlqr_tune_batched_set(ctypes.byref(bs), ctypes.byref(opts), route),
           "rlqr_tune_batched_set")
