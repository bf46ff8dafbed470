"""Sharded solve of one long-horizon instance over G ranks (one GPU each).

Rank g owns the contiguous stages [s_g, e_g] of the horizon and solves them
as an ordinary instance (a dynamic-programming cut) once three boundary
values are known: the cost-to-go (P_{e_g}, p_{e_g}) after the shard and
the state x_{s_g} at its start.  They come from three all-gathers of small
per-shard summaries (Section "Parallel Algorithm": interval elements of
contiguous stage ranges compose with the associative rule of eq.
lqr-gpu-combo; Corollary p-recurrence and Section "Composing Affine
Functions" for the p and x maps):

  1. the interval element (P, A, C) of the shard's stages      (3 n^2)
  2. the p map p_{s} = Phi p_{e} + phi of the factored shard    (n^2 + n)
  3. the offset psi of the x map x_{e} = Phi^T x_{s} + psi      (n)

Everything else is local to the rank.  The arithmetic runs in the library's
kernels (``rlqr_shard_*`` and the FP64 scan path); this module only places
boundary values in the shard's own arrays and moves summaries between ranks.
The compute steps are taken from an ``ops`` object (``CudaOps`` here), so
that the protocol can be exercised with other implementations of the same
steps.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable

import numpy as np
import torch

from . import rlqr


def shard_bounds(N: int, G: int) -> list[tuple[int, int]]:
    """Contiguous stage ranges [s_g, e_g] covering 0..N, sizes differing by at
    most one stage (every shard has at least one stage)."""
    if not 1 <= G <= N:
        raise ValueError("need 1 <= G <= N")
    cuts = [(g * N) // G for g in range(G + 1)]
    return [(cuts[g], cuts[g + 1]) for g in range(G)]


@dataclass
class ShardData:
    """One shard's arrays (stage-major FP64, the layout of rlqr_problem):
    Q, q, c hold stages s..e (N_g + 1 entries), M, R, r, A, B stages
    s..e-1.  Q[N_g], q[N_g] and c[0] are boundary slots; QN, qN are the
    instance's terminal Q_N, q_N (every rank needs them)."""
    g: int
    G: int
    s: int
    e: int
    n: int
    m: int
    delta: float
    Q: object
    M: object
    R: object
    q: object
    r: object
    A: object
    B: object
    c: object
    QN: object
    qN: object

    @property
    def N(self) -> int:
        return self.e - self.s

    @staticmethod
    def from_arrays(arrs: dict, N: int, n: int, m: int, delta: float, g: int, G: int,
                    to=lambda a: a) -> "ShardData":
        """Shard g of G from the full instance's stage-major arrays (numpy or
        torch); ``to`` converts each slice (e.g. to a contiguous CUDA
        tensor)."""
        s, e = shard_bounds(N, G)[g]

        def cut(k, a, b):
            v = arrs[k][a:b]
            return to(v.copy() if isinstance(v, np.ndarray) else v.clone())

        return ShardData(g, G, s, e, n, m, float(delta),
                         Q=cut("Q", s, e + 1), M=cut("M", s, e), R=cut("R", s, e),
                         q=cut("q", s, e + 1), r=cut("r", s, e), A=cut("A", s, e),
                         B=cut("B", s, e), c=cut("c", s, e + 1),
                         QN=cut("Q", N, N + 1)[0], qN=cut("q", N, N + 1)[0])


class HorizonShard:
    """The per-rank protocol.  Phases run in order; between them the caller
    gathers the returned summaries of all G shards (stacked in shard order).
    Afterwards ``x, u, y, flags`` hold the shard's part of the solution for
    its stages s..e (x, y, flags: N_g + 1 rows; row N_g equals row 0 of the
    next shard)."""

    def __init__(self, data: ShardData, ops):
        self.d, self.ops = data, ops
        self.last = data.g == data.G - 1
        self.c0 = data.c[0].clone() if hasattr(data.c, "clone") else data.c[0].copy()
        ops.setup(self.d)

    def phase_element(self):
        return self.ops.element(self.d)

    def phase_factor(self, elems):
        """P at the shard's end into its terminal slot, factor; returns the p
        map (Phi, phi) of a solve with a zero terminal p."""
        d, ops = self.d, self.ops
        self.P_end, self.P_start = ops.boundary(d, elems)
        if not self.last:
            d.Q[d.N] = self.P_end
        ops.factor(d)
        q_end = d.q[d.N].clone() if hasattr(d.q, "clone") else d.q[d.N].copy()
        d.q[d.N] = 0.0
        ops.solve(d)
        self.Phi, phi = ops.pmap(d)
        d.q[d.N] = q_end
        return self.Phi, phi

    def phase_offsets(self, Phis, phis):
        """p at the shard's end into its terminal slot, then a solve from
        c_0 = 0 (shard 0: its true c_0); returns the x-map offset psi."""
        d, ops = self.d, self.ops
        self.Phis = Phis
        if not self.last:
            d.q[d.N] = ops.p_end(d, Phis, phis)
        d.c[0] = self.c0 if d.g == 0 else 0.0
        ops.solve(d)
        x, _, _ = ops.solution(d)
        self.x_first = ops.zeros_like(x[0]) if d.g == 0 else x[0].clone() if hasattr(x, "clone") \
            else x[0].copy()
        return ops.x_offset(d, self.Phi, self.x_first, x[d.N])

    def phase_final(self, psis):
        """The initial term that starts the shard at the true x_{s_g}, and the
        final solve (shard 0's solve of the previous phase is final)."""
        d, ops = self.d, self.ops
        if d.g > 0:
            x_start = ops.x_start(d, self.Phis, psis)
            d.c[0] = ops.entry(d, self.P_start, x_start, self.x_first)
            ops.solve(d)
        return ops.solution(d)


def solve(shard: HorizonShard, gather: Callable):
    """Run the protocol on this rank; ``gather(t)`` returns the stacked
    tensors of all ranks (an all-gather)."""
    elems = gather(shard.phase_element())
    Phi, phi = shard.phase_factor(elems)
    Phis, phis = gather(Phi), gather(phi)
    psis = gather(shard.phase_offsets(Phis, phis))
    return shard.phase_final(psis)


def solve_lockstep(shards: list[HorizonShard]):
    """All G shards in one process, phase by phase (the gathers become
    stacks); for a single GPU or for checking the protocol."""
    elems = torch.stack([s.phase_element() for s in shards])
    maps = [s.phase_factor(elems) for s in shards]
    Phis = torch.stack([p for p, _ in maps])
    phis = torch.stack([f for _, f in maps])
    psis = torch.stack([s.phase_offsets(Phis, phis) for s in shards])
    return [s.phase_final(psis) for s in shards]


def torch_gather(group=None) -> Callable:
    """All-gather over torch.distributed (NCCL between GPUs, gloo on CPU)."""
    import torch.distributed as dist

    def gather(t):
        t = t.contiguous()
        out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
        dist.all_gather(out, t, group=group)
        return torch.stack(out)
    return gather


class CudaOps:
    """The shard steps through the library (FP64 associative-scan path)."""

    def __init__(self, max_refine: int = 0):
        self.opts = rlqr.make_opts(rlqr.RLQR_FP64, algo=rlqr.RLQR_ALGO_SCAN,
                                   max_refine=max_refine)

    def setup(self, d: ShardData):
        d._prob = rlqr.DeviceProblem(d.N, d.n, d.m, d.Q, d.M, d.R, d.q, d.r, d.A, d.B, d.c,
                                     d.delta)
        d._ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(d.N, d.n, d.m, self.opts))
        dev = d.Q.device
        d._x = torch.zeros(d.N + 1, d.n, dtype=torch.float64, device=dev)
        d._u = torch.zeros(d.N, d.m, dtype=torch.float64, device=dev)
        d._y = torch.zeros(d.N + 1, d.n, dtype=torch.float64, device=dev)
        d._flags = torch.zeros(d.N + 1, dtype=torch.uint8, device=dev)

    def element(self, d):
        elem = torch.empty(3, d.n, d.n, dtype=torch.float64, device=d.Q.device)
        rlqr.rlqr_shard_element(d._prob, self.opts, d._ws, elem)
        return elem

    def boundary(self, d, elems):
        P_end = torch.empty(d.n, d.n, dtype=torch.float64, device=d.Q.device)
        P_start = torch.empty_like(P_end)
        rlqr.rlqr_shard_boundary(d.G, d.g, d.n, d.m, elems.contiguous(), d.QN, P_end, P_start)
        return P_end, P_start

    def factor(self, d):
        rlqr.rlqr_factor(d._prob, self.opts, d._ws, d._flags)

    def solve(self, d):
        rlqr.rlqr_solve(d._prob, self.opts, d._ws, d._x, d._u, d._y)

    def pmap(self, d):
        Phi = torch.empty(d.n, d.n, dtype=torch.float64, device=d.Q.device)
        phi = torch.empty(d.n, dtype=torch.float64, device=d.Q.device)
        rlqr.rlqr_shard_pmap(d._prob, self.opts, d._ws, Phi, phi)
        return Phi, phi

    def p_end(self, d, Phis, phis):
        out = torch.empty(d.n, dtype=torch.float64, device=d.Q.device)
        rlqr.rlqr_shard_p_end(d.G, d.g, d.n, Phis.contiguous(), phis.contiguous(), d.qN, out)
        return out

    def x_offset(self, d, Phi, x_first, x_last):
        out = torch.empty(d.n, dtype=torch.float64, device=d.Q.device)
        rlqr.rlqr_shard_x_offset(d.n, Phi.contiguous(), x_first.contiguous(),
                                 x_last.contiguous(), out)
        return out

    def x_start(self, d, Phis, psis):
        out = torch.empty(d.n, dtype=torch.float64, device=d.Q.device)
        rlqr.rlqr_shard_x_start(d.g, d.n, Phis.contiguous(), psis.contiguous(), out)
        return out

    def entry(self, d, P_start, x_start, x_first):
        out = torch.empty(d.n, dtype=torch.float64, device=d.Q.device)
        rlqr.rlqr_shard_entry(d.n, d.delta, P_start, x_start, x_first.contiguous(), out)
        return out

    def solution(self, d):
        return d._x, d._u, d._y

    def flags(self, d):
        return d._flags

    @staticmethod
    def zeros_like(v):
        return torch.zeros_like(v)
