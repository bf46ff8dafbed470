"""The sharded long-horizon protocol on CPU ranks (gloo, world size 2 and 3).

paper_2509_16370_b300.shard runs the per-rank phases and the three
all-gathers over torch.distributed; here every compute step is the oracle's
(OracleShardOps: the interval elements and the combination rule of
oracle/scan.py, the sequential recursion of the C oracle for the shard's
sub-problem, and the affine maps written out in numpy), so the test checks
the protocol itself -- which boundary slots are written, what is gathered,
in which order the maps compose -- against the oracle's solution of the
whole horizon.  The same phases run through the CUDA library in
tests/test_gpu_shard.py.
"""
import os
import socket
import sys
from types import SimpleNamespace

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import scan as oscan  # noqa: E402
from paper_2509_16370_b300 import inputs, shard  # noqa: E402


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))


class OracleShardOps:
    """The shard steps restated with the oracle (FP64, host)."""

    def setup(self, d):
        d._res = None

    @staticmethod
    def _prob(d):
        return SimpleNamespace(N=d.N, n=d.n, m=d.m, delta=d.delta,
                               **{k: _np(getattr(d, k)) for k in ("Q", "M", "R", "q", "r", "A",
                                                                  "B", "c")})

    def element(self, d):
        sp = self._prob(d)
        e = oscan.stage_element(sp, 0)
        for i in range(1, d.N):
            e = oscan.combine(e, oscan.stage_element(sp, i))
        return _t(np.stack([e[0], e[2], e[3]]))

    def boundary(self, d, elems):
        n = d.n
        z, zv = np.zeros((n, n)), np.zeros(n)
        S = (_np(d.QN), _np(d.qN), z, z, zv)
        E = [(_np(el[0]), zv, _np(el[1]), _np(el[2]), zv) for el in elems]
        for h in range(d.G - 1, d.g, -1):
            S = oscan.combine(E[h], S)
        P_end = S[0]
        P_start = oscan.combine(E[d.g], S)[0]
        return _t(P_end), _t(P_start)

    def factor(self, d):
        pass  # the oracle factors and solves in one call (solve)

    def solve(self, d):
        sp = self._prob(d)
        d._res = oracle.riccati(sp, internals=True)
        d._sp = sp

    def pmap(self, d):
        sp, res = d._sp, d._res
        n = d.n
        I = np.eye(n)
        Phi = I
        for k in range(d.N):
            Wn = np.linalg.solve(I + d.delta * res.P[k + 1], res.P[k + 1])
            F = (sp.A[k] + sp.B[k] @ res.K[k]).T @ (I - d.delta * Wn)
            Phi = Phi @ F
        return _t(Phi), _t(res.p[0])

    def p_end(self, d, Phis, phis):
        v = _np(d.qN)
        for h in range(d.G - 1, d.g, -1):
            v = _np(Phis[h]) @ v + _np(phis[h])
        return _t(v)

    def x_offset(self, d, Phi, x_first, x_last):
        return _t(_np(x_last) - _np(Phi).T @ _np(x_first))

    def x_start(self, d, Phis, psis):
        v = _np(psis[0])
        for h in range(1, d.g):
            v = _np(Phis[h]).T @ v + _np(psis[h])
        return _t(v)

    def entry(self, d, P_start, x_start, x_first):
        P = _np(P_start)
        return _t((np.eye(d.n) + d.delta * P) @ (_np(x_start) - _np(x_first)))

    def solution(self, d):
        r = d._res
        return _t(r.x), _t(r.u), _t(r.y)

    def flags(self, d):
        return torch.from_numpy(d._res.flags.copy())

    @staticmethod
    def zeros_like(v):
        return torch.zeros_like(v)


def _instance():
    return inputs.random_instance(501, 47, 4, 2, 1e-2)


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _instance()
        arrs = {k: getattr(p, k) for k in ("Q", "M", "R", "q", "r", "A", "B", "c")}
        d = shard.ShardData.from_arrays(arrs, p.N, p.n, p.m, p.delta, rank, world, _t)
        hs = shard.HorizonShard(d, OracleShardOps())
        x, u, y = shard.solve(hs, shard.torch_gather())
        q.put((rank, d.s, d.e, _np(x), _np(u), _np(y), hs.ops.flags(d).numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_protocol_on_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = _instance()
    ref = oracle.riccati(p)
    xs, us, ys, fs = [], [], [], []
    for rank, s0, e0, x, u, y, f in res:
        L = e0 - s0
        keep = L + 1 if rank == world - 1 else L
        # the shard's rows are the whole horizon's rows s0 .. e0
        np.testing.assert_allclose(x, ref.x[s0:e0 + 1], rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(y, ref.y[s0:e0 + 1], rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(u, ref.u[s0:e0], rtol=1e-9, atol=1e-10)
        xs.append(x[:keep]), us.append(u), ys.append(y[:keep]), fs.append(f[:keep])
    x, u, y, f = map(np.concatenate, (xs, us, ys, fs))
    np.testing.assert_array_equal(f, ref.flags)
    assert oracle.residual(p, x, u, y).rel <= 1e-13


def test_shard_bounds_cover_the_horizon():
    for N in (1, 5, 47, 1000):
        for G in range(1, min(N, 7) + 1):
            b = shard.shard_bounds(N, G)
            assert b[0][0] == 0 and b[-1][1] == N and len(b) == G
            assert all(e0 == s1 for (_, e0), (s1, _) in zip(b[:-1], b[1:]))
            sizes = [e - s for s, e in b]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_bounds(3, 4)
