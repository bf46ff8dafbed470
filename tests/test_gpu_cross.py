"""Cross-stage variables on the GPU (Section "Cross-Stage Variables"):
rlqr_solve_cross against the oracle's dense bordered solve on the same
seeded inputs -- dw and dtheta, and the normwise backward error of the
bordered system computed on the host in FP64."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_16370_b300 import inputs, rlqr

pytestmark = pytest.mark.gpu


def _cross_inputs(seed, p, prob):
    rng = np.random.default_rng(seed)
    N, n, m = prob.N, prob.n, prob.m
    Jq = rng.standard_normal((p, N + 1, n))
    Jr = rng.standard_normal((p, N, m))
    Jc = 0.3 * rng.standard_normal((p, N + 1, n))
    Hs = rng.standard_normal((p, p))
    H = Hs + Hs.T + (2.0 * p) * np.eye(p)
    return Jq, Jr, Jc, H, rng.standard_normal(p)


def _gpu_cross(prob, prec, algo, Jq, Jr, Jc, H, rt, sync=False):
    dp = rlqr.DeviceProblem.from_host(prob)
    opts = rlqr.make_opts(prec, algo=algo, tol=1e-9, max_refine=4, sync=sync)
    N, n, m, p = prob.N, prob.n, prob.m, len(rt)
    ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(N, n, m, opts))
    flags = torch.zeros(N + 1, dtype=torch.uint8, device="cuda")
    rlqr.rlqr_factor(dp, opts, ws, flags)
    J = torch.from_numpy(np.concatenate([Jq.reshape(p, -1), Jr.reshape(p, -1), Jc.reshape(p, -1)],
                                        axis=1)).cuda().contiguous()
    scratch = rlqr.alloc_workspace(rlqr.rlqr_cross_scratch_bytes(N, n, m, p, opts))
    x = torch.zeros(N + 1, n, dtype=torch.float64, device="cuda")
    u = torch.zeros(N, m, dtype=torch.float64, device="cuda")
    y = torch.zeros(N + 1, n, dtype=torch.float64, device="cuda")
    dth = torch.zeros(p, dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    code = rlqr.rlqr_solve_cross(dp, opts, ws, J, torch.from_numpy(H).cuda(),
                                 torch.from_numpy(rt).cuda(), scratch, x, u, y, dth, st)
    torch.cuda.synchronize()
    return (code, int(st.item()), x.cpu().numpy(), u.cpu().numpy(), y.cpu().numpy(),
            dth.cpu().numpy())


def _bordered_backward_error(prob, Jq, Jr, Jc, H, rt, x, u, y, dth):
    K, b = oracle.kkt_dense(prob)
    p = len(rt)
    J = np.stack([oracle.join_solution(prob, Jq[j], Jr[j], Jc[j]) for j in range(p)], axis=1)
    big = np.block([[K, J], [J.T, H]])
    z = np.concatenate([oracle.join_solution(prob, x, u, y), dth])
    rhs = np.concatenate([b, rt])
    r = big @ z + rhs
    return np.abs(r).max() / (np.abs(big).sum(axis=1).max() * np.abs(z).max() + np.abs(rhs).max())


CASES = [(801, 20, 4, 2, 1e-3, 1, rlqr.RLQR_ALGO_SEQ), (802, 40, 12, 4, 1e-5, 3, rlqr.RLQR_ALGO_SEQ),
         (803, 33, 6, 2, 0.3, 2, rlqr.RLQR_ALGO_SEQ), (804, 64, 4, 2, 1e-2, 2, rlqr.RLQR_ALGO_SCAN),
         (805, 17, 24, 8, 1e-4, 4, rlqr.RLQR_ALGO_SEQ)]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[1]}n{c[2]}p{c[5]}a{c[6]}" for c in CASES])
@pytest.mark.parametrize("prec", [rlqr.RLQR_FP64, rlqr.RLQR_MIXED])
def test_cross_stage_matches_the_bordered_oracle(case, prec):
    seed, N, n, m, delta, p, algo = case
    prob = inputs.random_instance(seed, N, n, m, delta)
    Jq, Jr, Jc, H, rt = _cross_inputs(seed, p, prob)
    code, st, x, u, y, dth = _gpu_cross(prob, prec, algo, Jq, Jr, Jc, H, rt)
    assert code == rlqr.RLQR_OK and st in (rlqr.RLQR_OK, rlqr.RLQR_NOT_PD)
    rx, ru, ry, rth = oracle.cross_stage_solve(prob, Jq, Jr, Jc, H, rt)
    scale = max(np.abs(np.concatenate([rx.ravel(), ru.ravel(), ry.ravel(), rth])).max(), 1.0)
    tol = 1e-8 if prec == rlqr.RLQR_FP64 else 1e-6
    for got, ref in ((x, rx), (u, ru), (y, ry), (dth, rth)):
        assert np.abs(got - ref).max() <= tol * scale
    assert _bordered_backward_error(prob, Jq, Jr, Jc, H, rt, x, u, y, dth) <= 1e-9


@pytest.mark.parametrize("prec", [rlqr.RLQR_FP64, rlqr.RLQR_MIXED])
def test_cross_stage_singular_schur_complement(prec):
    """J = 0 and H = 0 make S = 0: RLQR_ERR_SINGULAR on the device, and as
    the host return with RLQR_OPT_SYNC; dtheta = 0, dw the plain solution."""
    prob = inputs.random_instance(806, 16, 4, 2, 1e-3)
    p = 2
    Z = lambda *s: np.zeros(s)  # noqa: E731
    for sync in (False, True):
        code, st, x, u, y, dth = _gpu_cross(prob, prec, rlqr.RLQR_ALGO_SEQ, Z(p, 17, 4),
                                            Z(p, 16, 2), Z(p, 17, 4), Z(p, p), np.ones(p),
                                            sync=sync)
        assert st == rlqr.RLQR_ERR_SINGULAR
        assert code == (rlqr.RLQR_ERR_SINGULAR if sync else rlqr.RLQR_OK)
        assert np.all(dth == 0.0)
        assert oracle.residual(prob, x, u, y).rel <= 1e-9


def test_cross_scratch_sizing():
    o = rlqr.make_opts(rlqr.RLQR_MIXED)
    assert rlqr.rlqr_cross_scratch_bytes(16, 4, 2, 0, o) == 0
    assert rlqr.rlqr_cross_scratch_bytes(16, 4, 2, 32, o) == 0
    a = rlqr.rlqr_cross_scratch_bytes(16, 4, 2, 1, o)
    b = rlqr.rlqr_cross_scratch_bytes(16, 4, 2, 4, o)
    assert 0 < a < b and a % 256 == 0


def test_cross_stage_graph_replay():
    """The p + 1 solves run on the library's own streams, forked from and
    joined back to the caller's stream: the call can be captured into a CUDA
    graph and a replay reproduces the eager result bit for bit."""
    prob = inputs.random_instance(807, 48, 12, 4, 1e-4)
    p = 3
    Jq, Jr, Jc, H, rt = _cross_inputs(807, p, prob)
    dp = rlqr.DeviceProblem.from_host(prob)
    opts = rlqr.make_opts(rlqr.RLQR_MIXED, algo=rlqr.RLQR_ALGO_SEQ, tol=1e-9, max_refine=4)
    N, n, m = prob.N, prob.n, prob.m
    ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(N, n, m, opts))
    flags = torch.zeros(N + 1, dtype=torch.uint8, device="cuda")
    rlqr.rlqr_factor(dp, opts, ws, flags)
    J = torch.from_numpy(np.concatenate([Jq.reshape(p, -1), Jr.reshape(p, -1), Jc.reshape(p, -1)],
                                        axis=1)).cuda().contiguous()
    Hd, rtd = torch.from_numpy(H).cuda(), torch.from_numpy(rt).cuda()
    scratch = rlqr.alloc_workspace(rlqr.rlqr_cross_scratch_bytes(N, n, m, p, opts))
    outs = [torch.zeros(N + 1, n, dtype=torch.float64, device="cuda"),
            torch.zeros(N, m, dtype=torch.float64, device="cuda"),
            torch.zeros(N + 1, n, dtype=torch.float64, device="cuda"),
            torch.zeros(p, dtype=torch.float64, device="cuda")]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        rlqr.rlqr_solve_cross(dp, opts, ws, J, Hd, rtd, scratch, *outs)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = [t.clone() for t in outs]
    for t in outs:
        t.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rlqr.rlqr_solve_cross(dp, opts, ws, J, Hd, rtd, scratch, *outs)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, outs):
        assert torch.equal(a, b)
