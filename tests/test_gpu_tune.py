"""Scan tiles and their autotuner (rlqr_autotune_scan): the associative
scan gives the oracle's flags and a backward error <= 1e-9 for every
candidate chunk count (148 .. 888 chunks, the tiles the autotuner chooses
among), both precisions; the autotuner returns one of them and the solves
after it stay exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_16370_b300 import inputs, rlqr

pytestmark = pytest.mark.gpu


def _bufs(p):
    f = dict(dtype=torch.float64, device="cuda")
    return (torch.zeros(p.N + 1, p.n, **f), torch.zeros(p.N, p.m, **f),
            torch.zeros(p.N + 1, p.n, **f), torch.zeros(p.N + 1, dtype=torch.uint8, device="cuda"))


def _check(p, ref, x, u, y, flags):
    np.testing.assert_array_equal(flags.cpu().numpy(), ref.flags)
    r = oracle.residual(p, x.cpu().numpy(), u.cpu().numpy(), y.cpu().numpy()).rel
    assert r <= 1e-9, r


@pytest.mark.parametrize("prec", [rlqr.RLQR_FP64, rlqr.RLQR_MIXED])
def test_every_chunk_count_is_exact(prec):
    p = inputs.random_instance(91, 6000, 12, 4, 1e-4)
    ref = oracle.riccati(p)
    dp = rlqr.DeviceProblem.from_host(p)
    opts = rlqr.make_opts(prec, algo=rlqr.RLQR_ALGO_SCAN, tol=1e-9, max_refine=4)
    ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(p.N, p.n, p.m, opts))
    x, u, y, flags = _bufs(p)
    try:
        for chunks in rlqr.SCAN_CHUNK_CANDIDATES + (37,):
            rlqr.rlqr_tune_scan_set(p.N, p.n, p.m, opts, chunks)
            rlqr.rlqr_factor(dp, opts, ws, flags)
            rlqr.rlqr_solve(dp, opts, ws, x, u, y)
            torch.cuda.synchronize()
            _check(p, ref, x, u, y, flags)
    finally:
        rlqr.rlqr_tune_reset()


def test_autotuner_choice_and_solves_after_it():
    p = inputs.random_instance(92, 8192, 12, 4, 1e-4)
    ref = oracle.riccati(p)
    dp = rlqr.DeviceProblem.from_host(p)
    opts = rlqr.make_opts(rlqr.RLQR_MIXED, algo=rlqr.RLQR_ALGO_SCAN, tol=1e-9, max_refine=4)
    ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(p.N, p.n, p.m, opts))
    x, u, y, flags = _bufs(p)
    try:
        chunks, ms = rlqr.rlqr_autotune_scan(dp, opts, ws, x, u, y, flags)
        assert chunks in rlqr.SCAN_CHUNK_CANDIDATES and ms > 0
        x.zero_()
        rlqr.rlqr_factor(dp, opts, ws, flags)
        rlqr.rlqr_solve(dp, opts, ws, x, u, y)
        torch.cuda.synchronize()
        _check(p, ref, x, u, y, flags)
        # a shape the scan does not take: rejected before any work
        q = inputs.random_instance(93, 64, 5, 2, 1e-4)
        with pytest.raises(rlqr.RlqrError):
            rlqr.rlqr_autotune_scan(rlqr.DeviceProblem.from_host(q), opts, ws, *_bufs(q))
    finally:
        rlqr.rlqr_tune_reset()


@pytest.mark.parametrize("prec,nm", [(rlqr.RLQR_FP64, (12, 4)), (rlqr.RLQR_MIXED, (12, 4)),
                                     (rlqr.RLQR_MIXED, (6, 1))])
def test_every_batched_residual_route_is_exact_and_the_tuner_picks_one(prec, nm):
    """Routes 1 (warp residual), 2 (grid residual) and, mixed, 5 (the first
    refinement pass computes the residual itself), 6 and 7 (routes 1 and 5
    with the refinement passes on two warps per instance): the oracle's flags, its
    backward error <= 1e-9 for every instance, the reported backward error
    an upper bound of the oracle's, the same statuses on every route."""
    from tests.gpu_helpers import REL_TOL
    n, m = nm
    probs = [inputs.random_instance(300 + b, 96 + 8 * (b % 5), n, m, 1e-3) for b in range(64)]
    probs[7].Q[20] -= 3.0 * np.eye(n)  # a non-PD pivot somewhere in the batch
    db = rlqr.DeviceBatch.from_problems(probs)
    opts = rlqr.make_opts(prec, tol=1e-9, max_refine=4)
    ws = rlqr.alloc_workspace(rlqr.rlqr_batched_workspace_bytes(db, opts))
    st = torch.zeros(db.count, dtype=torch.int32, device="cuda")
    rel = torch.zeros(db.count, dtype=torch.float64, device="cuda")
    refs = [oracle.riccati(p) for p in probs]
    routes = [rlqr.RES_ROUTE_WARP, rlqr.RES_ROUTE_GRID]
    if prec == rlqr.RLQR_MIXED:
        routes += [rlqr.RES_ROUTE_FUSED, rlqr.RES_ROUTE_WARP_DUO, rlqr.RES_ROUTE_FUSED_DUO]
    statuses = []
    try:
        for route in routes:
            rlqr.rlqr_tune_batched_set(db, opts, route)
            rlqr.rlqr_solve_batched(db, opts, ws, st, rel)
            torch.cuda.synchronize()
            rels = rel.cpu().numpy()
            for b, p in enumerate(probs):
                x, u, y, f = db.instance_view(b)
                np.testing.assert_array_equal(f, refs[b].flags, err_msg=f"route {route} {b}")
                r = oracle.residual(p, x, u, y).rel
                assert r <= REL_TOL, (route, b, r)
                assert rels[b] <= REL_TOL and r <= 1.05 * rels[b] + 1e-15, (route, b, r, rels[b])
            statuses.append(st.cpu().numpy().copy())
        for sv in statuses[1:]:
            np.testing.assert_array_equal(sv, statuses[0])
        route, ms = rlqr.rlqr_autotune_batched(db, opts, ws, st)
        assert route in routes and ms > 0
        if prec == rlqr.RLQR_FP64:
            for r in (rlqr.RES_ROUTE_FUSED, rlqr.RES_ROUTE_WARP_DUO, rlqr.RES_ROUTE_FUSED_DUO):
                with pytest.raises(rlqr.RlqrError):
                    rlqr.rlqr_tune_batched_set(db, opts, r)
    finally:
        rlqr.rlqr_tune_reset()
