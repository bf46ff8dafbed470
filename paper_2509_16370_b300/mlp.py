"""Thin ctypes binding of include/rlqr_mlp.h (the IPM warm-start network) and
the warm-start helpers around it.

Marshalling only: the forward pass, the gradient and the Adam step run in the
CUDA kernels of librlqr.so.  ``WarmStartNet`` holds the parameters (FP32
master, BF16 copy, Adam moments) as torch CUDA tensors; ``train`` loops over
shuffled mini-batches calling rlqr_mlp_grad and rlqr_mlp_adam; ``propose``
maps (x0, goal) to an initial trajectory (X, U) for rlqr_ipm_init.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from .rlqr import _check, _ptr, _stream, lib

EXPORTED = ("rlqr_mlp_param_count", "rlqr_mlp_workspace_bytes", "rlqr_mlp_sync_bf16",
            "rlqr_mlp_forward", "rlqr_mlp_grad", "rlqr_mlp_adam", "rlqr_mlp_train_step")


class rlqr_mlp_dims(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("width", ctypes.c_int32), ("n_out", ctypes.c_int32),
                ("max_rows", ctypes.c_int32)]


_P, _dp, _i, _f = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int32, ctypes.c_float
lib.rlqr_mlp_param_count.restype = ctypes.c_size_t
lib.rlqr_mlp_param_count.argtypes = [_P(rlqr_mlp_dims)]
lib.rlqr_mlp_workspace_bytes.restype = ctypes.c_size_t
lib.rlqr_mlp_workspace_bytes.argtypes = [_P(rlqr_mlp_dims)]
lib.rlqr_mlp_sync_bf16.restype = ctypes.c_int
lib.rlqr_mlp_sync_bf16.argtypes = [_P(rlqr_mlp_dims), _dp, _dp, _dp]
lib.rlqr_mlp_forward.restype = ctypes.c_int
lib.rlqr_mlp_forward.argtypes = [_P(rlqr_mlp_dims), _dp, _dp, _i, _dp, _dp, ctypes.c_size_t, _dp]
lib.rlqr_mlp_grad.restype = ctypes.c_int
lib.rlqr_mlp_grad.argtypes = [_P(rlqr_mlp_dims), _dp, _dp, _dp, _dp, _i, _dp, _dp, _dp,
                              ctypes.c_size_t, _dp]
lib.rlqr_mlp_adam.restype = ctypes.c_int
lib.rlqr_mlp_adam.argtypes = [_P(rlqr_mlp_dims), _dp, _dp, _dp, _dp, _dp, _i, _f, _f, _f, _f, _dp]
lib.rlqr_mlp_train_step.restype = ctypes.c_int
lib.rlqr_mlp_train_step.argtypes = [_P(rlqr_mlp_dims), _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _i,
                                    _dp, _dp, _f, _f, _f, _dp, _dp, ctypes.c_size_t, _dp]


def make_dims(n_in, width, n_out, max_rows) -> rlqr_mlp_dims:
    return rlqr_mlp_dims(n_in, width, n_out, max_rows)


def rlqr_mlp_param_count(d) -> int:
    return int(lib.rlqr_mlp_param_count(ctypes.byref(d)))


def rlqr_mlp_workspace_bytes(d) -> int:
    return int(lib.rlqr_mlp_workspace_bytes(ctypes.byref(d)))


class WarmStartNet:
    """Parameters, BF16 copy, Adam moments and workspace of one network."""

    def __init__(self, d: rlqr_mlp_dims, params: np.ndarray, device="cuda"):
        self.d = d
        n = rlqr_mlp_param_count(d)
        assert params.size == n
        self.p = torch.from_numpy(np.asarray(params, np.float32)).to(device)
        self.q = torch.zeros(n, dtype=torch.int16, device=device)   # BF16 bit patterns
        self.m = torch.zeros(n, dtype=torch.float32, device=device)
        self.v = torch.zeros(n, dtype=torch.float32, device=device)
        self.g = torch.zeros(n, dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.ws = torch.empty(rlqr_mlp_workspace_bytes(d), dtype=torch.uint8, device=device)
        self.step = 0
        _check(lib.rlqr_mlp_sync_bf16(ctypes.byref(d), _ptr(self.p), _ptr(self.q),
                                      _stream(None)), "rlqr_mlp_sync_bf16")

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        rows = x.shape[0]
        y = torch.empty(rows, self.d.n_out, dtype=torch.float32, device=x.device)
        _check(lib.rlqr_mlp_forward(ctypes.byref(self.d), _ptr(self.q), _ptr(x), rows, _ptr(y),
                                    _ptr(self.ws), self.ws.numel(), _stream(None)),
               "rlqr_mlp_forward")
        return y

    def grad(self, x, t, idx):
        _check(lib.rlqr_mlp_grad(ctypes.byref(self.d), _ptr(self.q), _ptr(x), _ptr(t), _ptr(idx),
                                 idx.numel(), _ptr(self.loss), _ptr(self.g), _ptr(self.ws),
                                 self.ws.numel(), _stream(None)), "rlqr_mlp_grad")
        return self.loss, self.g

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.step += 1
        _check(lib.rlqr_mlp_adam(ctypes.byref(self.d), _ptr(self.p), _ptr(self.q), _ptr(self.m),
                                 _ptr(self.v), _ptr(self.g), self.step, lr, b1, b2, eps,
                                 _stream(None)), "rlqr_mlp_adam")

    def train_step(self, x, t, idx_all, rows, counter, sched, b1=0.9, b2=0.999, eps=1e-8):
        """One step of a device-scheduled sequence (rlqr_mlp_train_step); the
        caller advances self.step by the steps it replays."""
        _check(lib.rlqr_mlp_train_step(ctypes.byref(self.d), _ptr(self.p), _ptr(self.q),
                                       _ptr(self.m), _ptr(self.v), _ptr(self.g), _ptr(x), _ptr(t),
                                       _ptr(idx_all), rows, _ptr(counter), _ptr(sched), b1, b2,
                                       eps, _ptr(self.loss), _ptr(self.ws), self.ws.numel(),
                                       _stream(None)), "rlqr_mlp_train_step")


def save_checkpoint(net: WarmStartNet, path: str) -> None:
    """Training state of `net` to an .npz file: the FP32 parameters, the Adam
    moments, the step counter (the bias correction's t) and the dimensions.
    The BF16 copy is not stored: it is the rounding of the parameters and is
    rebuilt on load."""
    d = net.d
    np.savez(path, p=net.p.cpu().numpy(), m=net.m.cpu().numpy(), v=net.v.cpu().numpy(),
             step=np.int64(net.step),
             dims=np.array([d.n_in, d.width, d.n_out, d.max_rows], np.int64))


def load_checkpoint(path: str, device="cuda") -> WarmStartNet:
    """A network restored from save_checkpoint: training continues from it as
    from the saved network (same parameters, moments and step counter, so the
    next Adam steps are bit-identical)."""
    z = np.load(path)
    n_in, width, n_out, max_rows = (int(v) for v in z["dims"])
    net = WarmStartNet(make_dims(n_in, width, n_out, max_rows), z["p"], device=device)
    net.m.copy_(torch.from_numpy(z["m"]).to(device))
    net.v.copy_(torch.from_numpy(z["v"]).to(device))
    net.step = int(z["step"])
    return net


def init_params(d: rlqr_mlp_dims, seed: int) -> np.ndarray:
    """He-uniform weights, zero biases, zero padding (host, seeded)."""
    rng = np.random.default_rng(seed)
    W, npad = d.width, (d.n_out + 15) // 16 * 16
    parts = []
    W1 = np.zeros((W, 16))
    W1[:, :d.n_in] = rng.uniform(-1, 1, (W, d.n_in)) * np.sqrt(6.0 / d.n_in)
    W2 = rng.uniform(-1, 1, (W, W)) * np.sqrt(6.0 / W)
    W3 = np.zeros((npad, W))
    W3[:d.n_out] = rng.uniform(-1, 1, (d.n_out, W)) * np.sqrt(3.0 / W)
    for a in (W1, np.zeros(W), W2, np.zeros(W), W3, np.zeros(npad)):
        parts.append(a.ravel())
    return np.concatenate(parts).astype(np.float32)


def train(net: WarmStartNet, x: torch.Tensor, t: torch.Tensor, steps: int, batch: int,
          lr: float, seed: int = 0, lr_final: float | None = None) -> list:
    """Mini-batch Adam on (x, t) (device FP32 tensors); the shuffled index
    batches come from a seeded host permutation.  Returns the loss every 100
    steps."""
    n = x.shape[0]
    g = torch.Generator().manual_seed(seed)
    losses, perm, at = [], torch.randperm(n, generator=g), 0
    for s in range(steps):
        if at + batch > n:
            perm, at = torch.randperm(n, generator=g), 0
        idx = perm[at:at + batch].to(torch.int32).to(x.device)
        at += batch
        loss, _ = net.grad(x, t, idx)
        rate = lr if lr_final is None else lr * (lr_final / lr) ** (s / max(steps - 1, 1))
        net.adam(rate)
        if s % 100 == 0 or s == steps - 1:
            losses.append(float(loss.item()))
    return losses


def train_schedule(n: int, steps: int, batch: int, lr: float, seed: int = 0,
                   lr_final: float | None = None, step0: int = 0, b1: float = 0.9,
                   b2: float = 0.999):
    """The batches and Adam constants of train()'s steps, on the host: int32
    indices [steps][batch] (the same seeded permutations) and FP32 (lr, 1 -
    b1^t, 1 - b2^t) [steps][3], t = step0 + s + 1 (the C library's powf, as
    rlqr_mlp_adam forms them on the host)."""
    powf = _libm_powf()
    g = torch.Generator().manual_seed(seed)
    perm, at = torch.randperm(n, generator=g), 0
    idx = np.empty((steps, batch), np.int32)
    sched = np.empty((steps, 3), np.float32)
    one = np.float32(1.0)
    for s in range(steps):
        if at + batch > n:
            perm, at = torch.randperm(n, generator=g), 0
        idx[s] = perm[at:at + batch].numpy()
        at += batch
        rate = lr if lr_final is None else lr * (lr_final / lr) ** (s / max(steps - 1, 1))
        tt = float(step0 + s + 1)
        sched[s] = (np.float32(rate), one - np.float32(powf(b1, tt)),
                    one - np.float32(powf(b2, tt)))
    return idx, sched


def _libm_powf():
    libm = ctypes.CDLL("libm.so.6")
    libm.powf.restype = ctypes.c_float
    libm.powf.argtypes = [ctypes.c_float, ctypes.c_float]
    return libm.powf


def train_graph(net: WarmStartNet, x: torch.Tensor, t: torch.Tensor, steps: int, batch: int,
                lr: float, seed: int = 0, lr_final: float | None = None) -> list:
    """train(), with the whole step (gradient and Adam: 19 launches) captured
    once into a CUDA graph and replayed; the batches and the learning-rate
    schedule are read on the device.  The same kernels on the same inputs:
    the parameters equal train()'s.  Returns the loss every 100 steps."""
    idx, sched = train_schedule(x.shape[0], steps, batch, lr, seed, lr_final, net.step)
    idx_d = torch.from_numpy(idx).to(x.device)
    sched_d = torch.from_numpy(sched).to(x.device)
    counter = torch.zeros(1, dtype=torch.int32, device=x.device)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        net.train_step(x, t, idx_d, batch, counter, sched_d)
    losses = []
    for s in range(steps):
        graph.replay()
        if s % 100 == 0 or s == steps - 1:
            losses.append(float(net.loss.item()))
    net.step += steps
    return losses


# ---- warm start of the cart-double-pendulum IPM
N_IN = 7          # x0 (6) and the goal cart position


def features(x0: np.ndarray, xg: np.ndarray) -> np.ndarray:
    """Network input of each instance: its initial state and goal position."""
    return np.concatenate([x0, xg[:, :1]], axis=1).astype(np.float32)


def targets(X: np.ndarray, U: np.ndarray) -> np.ndarray:
    """Network output of each instance: its state trajectory and controls."""
    return np.concatenate([X.reshape(X.shape[0], -1), U], axis=1)


class Normalizer:
    """Per-column mean and standard deviation of the training targets."""

    def __init__(self, T: np.ndarray):
        self.mean = T.mean(axis=0)
        self.std = np.maximum(T.std(axis=0), 1e-6)

    def encode(self, T):
        return ((T - self.mean) / self.std).astype(np.float32)

    def decode(self, Y):
        return Y * self.std + self.mean


def propose(net: WarmStartNet, norm: Normalizer, x0: np.ndarray, xg: np.ndarray, N: int):
    """Initial trajectories (X [count][N+1][6], U [count][N], FP64 device
    tensors) for rlqr_ipm_init, in chunks of the network's max_rows."""
    count = x0.shape[0]
    feats = torch.from_numpy(features(x0, xg)).cuda()
    R = net.d.max_rows
    outs = []
    for s in range(0, count, R):
        n = min(R, count - s)
        rows = (n + 15) // 16 * 16
        chunk = torch.zeros(rows, N_IN, dtype=torch.float32, device="cuda")
        chunk[:n] = feats[s:s + n]
        outs.append(net.forward(chunk)[:n])
    Y = norm.decode(torch.cat(outs).double().cpu().numpy())
    X = Y[:, :(N + 1) * 6].reshape(count, N + 1, 6)
    X[:, 0] = x0                       # the initial state is known exactly
    U = Y[:, (N + 1) * 6:]
    return torch.from_numpy(np.ascontiguousarray(X)).cuda(), \
        torch.from_numpy(np.ascontiguousarray(U)).cuda()
