"""Sharded long-horizon solve on one GPU: G shards of one instance run the
per-rank protocol of paper_2509_16370_b300.shard in lockstep (the gathers
become stacks), every step through the library's kernels.  The assembled
solution is checked against the oracle's sequential recursion on the whole
horizon: flags byte-identical, forward error and backward error at FP64
level; the shard summaries against the oracle's interval elements."""
import numpy as np
import pytest
import torch

import oracle
from oracle import scan as oscan
from paper_2509_16370_b300 import inputs, rlqr, shard

pytestmark = pytest.mark.gpu


def _shards(p, G):
    arrs = {k: getattr(p, k) for k in ("Q", "M", "R", "q", "r", "A", "B", "c")}
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    ops = shard.CudaOps()
    return [shard.HorizonShard(shard.ShardData.from_arrays(arrs, p.N, p.n, p.m, p.delta, g, G,
                                                           to), ops) for g in range(G)]


def _assemble(shards, outs):
    xs, us, ys, fs = [], [], [], []
    for hs, (x, u, y) in zip(shards, outs):
        L = hs.d.N
        keep = L + 1 if hs.last else L
        xs.append(x[:keep].cpu().numpy())
        ys.append(y[:keep].cpu().numpy())
        us.append(u[:L].cpu().numpy())
        fs.append(hs.ops.flags(hs.d)[:keep].cpu().numpy())
    return np.concatenate(xs), np.concatenate(us), np.concatenate(ys), np.concatenate(fs)


CASES = [(401, 300, 4, 2, 1e-3), (402, 257, 12, 4, 1e-5), (403, 520, 6, 2, 0.3),
         (404, 640, 32, 8, 1e-7)]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[1]}n{c[2]}m{c[3]}" for c in CASES])
@pytest.mark.parametrize("G", [1, 2, 3, 5])
def test_sharded_solution_matches_oracle(case, G):
    seed, N, n, m, delta = case
    p = inputs.random_instance(seed, N, n, m, delta)
    shards = _shards(p, G)
    outs = shard.solve_lockstep(shards)
    torch.cuda.synchronize()
    # neighbouring shards agree on the shared boundary stage
    for a, b in zip(outs[:-1], outs[1:]):
        na = a[0].shape[0] - 1
        np.testing.assert_allclose(a[0][na].cpu().numpy(), b[0][0].cpu().numpy(),
                                   rtol=1e-9, atol=1e-9)
    x, u, y, f = _assemble(shards, outs)
    ref = oracle.riccati(p)
    np.testing.assert_array_equal(f, ref.flags)
    assert oracle.forward_error((ref.x, ref.u, ref.y), x, u, y) <= 1e-9
    # the FP64 scan alone (G = 1) reaches ~5e-12 at n = 32 (its eliminations
    # of I + C P); sharding adds three summaries and must stay far below the
    # 1e-9 target
    assert oracle.residual(p, x, u, y).rel <= 1e-10


def test_shard_element_and_boundary_match_the_oracle_fold():
    """rlqr_shard_element = the left-to-right composition of the shard's stage
    elements; rlqr_shard_boundary's P_end / P_start = the sequential P at
    the shard's end / start."""
    p = inputs.random_instance(405, 90, 4, 2, 1e-2)
    G = 3
    shards = _shards(p, G)
    elems = torch.stack([s.phase_element() for s in shards])
    torch.cuda.synchronize()
    P_seq = oracle.riccati(p, internals=True).P
    for g, hs in enumerate(shards):
        s0, e0 = hs.d.s, hs.d.e
        e = oscan.stage_element(p, s0)
        for i in range(s0 + 1, e0):
            e = oscan.combine(e, oscan.stage_element(p, i))
        got = elems[g].cpu().numpy()
        for k, ref in ((0, e[0]), (1, e[2]), (2, e[3])):
            np.testing.assert_allclose(got[k], ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
        P_end, P_start = hs.ops.boundary(hs.d, elems)
        np.testing.assert_allclose(P_end.cpu().numpy(), P_seq[e0], rtol=1e-10,
                                   atol=1e-10 * np.abs(P_seq[e0]).max())
        np.testing.assert_allclose(P_start.cpu().numpy(), P_seq[s0], rtol=1e-10,
                                   atol=1e-10 * np.abs(P_seq[s0]).max())


def test_shard_calls_reject_what_they_do_not_support():
    p = inputs.random_instance(406, 20, 4, 2, 1e-2)
    d = shard.ShardData.from_arrays({k: getattr(p, k) for k in ("Q", "M", "R", "q", "r", "A",
                                                                "B", "c")}, p.N, p.n, p.m,
                                    p.delta, 0, 1,
                                    lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda())
    prob = rlqr.DeviceProblem(d.N, d.n, d.m, d.Q, d.M, d.R, d.q, d.r, d.A, d.B, d.c, d.delta)
    elem = torch.empty(3, 4, 4, dtype=torch.float64, device="cuda")
    mixed = rlqr.make_opts(rlqr.RLQR_MIXED, algo=rlqr.RLQR_ALGO_SCAN)
    ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(d.N, 4, 2, mixed))
    with pytest.raises(rlqr.RlqrError, match="argument"):
        rlqr.rlqr_shard_element(prob, mixed, ws, elem)           # FP64 only
    fp64 = rlqr.make_opts(rlqr.RLQR_FP64, algo=rlqr.RLQR_ALGO_SCAN)
    small = rlqr.alloc_workspace(64)
    with pytest.raises(rlqr.RlqrError, match="workspace"):
        rlqr.rlqr_shard_element(prob, fp64, small, elem)
    P = torch.empty(4, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(rlqr.RlqrError, match="argument"):
        rlqr.rlqr_shard_boundary(2, 2, 4, 2, elem, P, P)         # g out of range
