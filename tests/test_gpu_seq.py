"""GPU parity of the sequential Riccati path against the FP64 oracle, through
the C ABI (rlqr_factor / rlqr_solve / rlqr_residual / rlqr_solve_batched)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2509_16370_b300 import inputs
from paper_2509_16370_b300 import rlqr
from tests.gpu_helpers import (FWD_TOL, REL_TOL, check_against_oracle, solve_batch, solve_single,
                               workload4_item, workload4_oracle_flags)

pytestmark = pytest.mark.gpu
PRECS = [rlqr.RLQR_FP64, rlqr.RLQR_MIXED]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        d = json.load(f)
    arr = {k: np.array(d[k], dtype=np.float64) for k in ("Q", "M", "R", "q", "r", "A", "B", "c")}
    return d, inputs.Problem(d["N"], d["n"], d["m"], delta=float(d["delta"]), **arr)


@pytest.mark.parametrize("prec", PRECS)
def test_workload1_single_instance(prec):
    """n=4, m=2, N=64, delta=1e-6: flags identical, rel-resid <= 1e-9, and the
    dense Bunch-Kaufman solution of the full KKT system agrees."""
    p = inputs.workload1()
    out = solve_single(p, prec)
    rel, fe, ref = check_against_oracle(p, out, prec)
    assert out["status"] == rlqr.RLQR_OK and out["status_factor"] == rlqr.RLQR_OK
    x, u, y, inertia = oracle.dense_solve(p)
    assert oracle.forward_error((x, u, y), out["x"], out["u"], out["y"]) <= FWD_TOL[prec]
    nxp, nyd = oracle.kkt_dims(p.N, p.n, p.m)
    assert inertia == (nxp, nyd, 0) and (out["flags"] == 3).all()
    # the GPU's own residual agrees with the oracle's (the mixed path updates it
    # with FP32 products of the corrections: ~1e-12 absolute)
    want = oracle.residual(p, out["x"], out["u"], out["y"]).rel
    if prec == rlqr.RLQR_FP64:
        assert out["rel"] == pytest.approx(want, rel=1e-3, abs=1e-15)
    else:
        assert out["rel"] == pytest.approx(want, rel=0.05, abs=1e-11)


@pytest.mark.parametrize("prec", PRECS)
def test_worked_examples(prec):
    d, p = _golden("worked_example_1.json")
    out = solve_single(p, prec)
    z = oracle.join_solution(p, out["x"], out["u"], out["y"])
    np.testing.assert_allclose(z, d["printed_solution"]["value"], atol=1e-12)
    d, p = _golden("worked_example_2.json")
    out = solve_single(p, prec)
    check_against_oracle(p, out, prec)
    assert list(out["flags"]) == [3, 3]


CASES = [  # (seed, N, n, m, delta, with_M) spanning every kernel bucket and ragged tails
    (1, 1, 1, 1, 1e-3, True), (2, 2, 3, 1, 0.0, True), (3, 7, 4, 2, 1e-2, True),
    (4, 33, 8, 4, 1e-6, True), (5, 5, 9, 3, 0.5, True), (6, 17, 12, 4, 1e-8, False),
    (7, 9, 16, 8, 1e-4, True), (8, 6, 17, 5, 1e-3, True), (9, 4, 32, 16, 1e-2, True),
    (10, 3, 33, 11, 1e-5, True), (11, 3, 48, 16, 1e-7, True), (12, 40, 6, 2, 2.0, True),
    (13, 21, 6, 1, 1e-3, True), (14, 19, 24, 8, 1e-4, True), (15, 11, 32, 8, 1e-6, True),
    # the FP32 tableau sweep's sizes with odd control dimensions and short horizons
    (16, 9, 4, 1, 1e-3, True), (17, 30, 12, 3, 1e-5, True), (18, 1, 12, 4, 1e-2, True),
    (19, 2, 6, 2, 1e-4, True), (20, 3, 4, 2, 1e-6, True), (21, 64, 6, 1, 1e-7, False)]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[1]}n{c[2]}m{c[3]}" for c in CASES])
@pytest.mark.parametrize("prec", PRECS)
def test_random_instances(case, prec):
    seed, N, n, m, delta, withM = case
    p = inputs.random_instance(seed, N, n, m, delta, with_M=withM)
    out = solve_single(p, prec)
    check_against_oracle(p, out, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_nonconvex_and_indefinite_pivots(prec):
    """Indefinite stage Hessians with nonsingular KKT: flags report the failing
    pivots exactly and the solution is still the KKT solution (Theorem
    riccati-rational-identity-theorem)."""
    p = inputs.random_instance(77, 12, 3, 2, 0.3, with_M=True)
    p.Q[4] -= 4.0 * np.eye(3)
    p.R[7] -= 3.0 * np.eye(2)
    ref = oracle.riccati(p)
    assert ref.status == oracle.NOT_PD
    out = solve_single(p, prec)
    check_against_oracle(p, out, prec)
    assert out["status_factor"] == rlqr.RLQR_NOT_PD


@pytest.mark.parametrize("prec", PRECS)
def test_singular_pivot_reports_status(prec):
    """I + delta P_1 = 1 + (-1) = 0: the recursion is undefined; the library
    reports RLQR_ERR_SINGULAR and returns normally."""
    p = inputs.Problem(1, 1, 1, Q=np.array([[[1.0]], [[-1.0]]]), M=np.zeros((1, 1, 1)),
                       R=np.array([[[1.0]]]), q=np.ones((2, 1)), r=np.ones((1, 1)),
                       A=np.ones((1, 1, 1)), B=np.ones((1, 1, 1)), c=np.ones((2, 1)), delta=1.0)
    out = solve_single(p, prec)
    assert out["status_factor"] == rlqr.RLQR_ERR_SINGULAR
    assert out["status"] == rlqr.RLQR_ERR_SINGULAR


@pytest.mark.parametrize("prec", PRECS)
def test_factor_reuse_for_new_rhs(prec):
    """Corollary p-recurrence: one factorization serves several right-hand sides."""
    p = inputs.random_instance(90, 20, 5, 2, 1e-3)
    out = solve_single(p, prec)
    check_against_oracle(p, out, prec)
    rng = np.random.default_rng(3)
    for _ in range(2):
        p.q = rng.standard_normal(p.q.shape)
        p.r = rng.standard_normal(p.r.shape)
        p.c = rng.standard_normal(p.c.shape)
        dp = rlqr.DeviceProblem.from_host(p)
        x = torch.zeros(p.N + 1, p.n, dtype=torch.float64, device="cuda")
        u = torch.zeros(p.N, p.m, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        rel = torch.zeros(1, dtype=torch.float64, device="cuda")
        rlqr.rlqr_solve(dp, out["opts"], out["ws"], x, u, y, rel)
        torch.cuda.synchronize()
        o2 = dict(x=x.cpu().numpy(), u=u.cpu().numpy(), y=y.cpu().numpy(), flags=out["flags"])
        check_against_oracle(p, o2, prec)


def test_residual_matches_oracle():
    p = inputs.random_instance(91, 15, 6, 3, 0.2)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((p.N + 1, p.n))
    u = rng.standard_normal((p.N, p.m))
    y = rng.standard_normal((p.N + 1, p.n))
    dp = rlqr.DeviceProblem.from_host(p)
    tx, tu, ty = (torch.from_numpy(a).cuda() for a in (x, u, y))
    dim = (p.N + 1) * p.n * 2 + p.N * p.m
    res = torch.zeros(dim, dtype=torch.float64, device="cuda")
    norms = torch.zeros(5, dtype=torch.float64, device="cuda")
    rlqr.rlqr_residual(dp, tx, tu, ty, res, norms)
    torch.cuda.synchronize()
    ref = oracle.residual(p, x, u, y)
    want = np.concatenate([ref.res_q.ravel(), ref.res_r.ravel(), ref.res_c.ravel()])
    np.testing.assert_allclose(res.cpu().numpy(), want, rtol=1e-13, atol=1e-13)
    nv = norms.cpu().numpy()
    np.testing.assert_allclose(nv[[0, 2, 3]], [ref.rmax, ref.zmax, ref.bmax], rtol=1e-12)
    # ||K||_inf is summed in FP32 on the device (it only scales the backward error)
    np.testing.assert_allclose(nv[[1, 4]], [ref.kmax, ref.rel], rtol=1e-5)


def test_workspace_errors():
    p = inputs.random_instance(92, 4, 3, 1, 1e-3)
    dp = rlqr.DeviceProblem.from_host(p)
    opts = rlqr.make_opts(rlqr.RLQR_FP64)
    nb = rlqr.rlqr_workspace_bytes(p.N, p.n, p.m, opts)
    small = rlqr.alloc_workspace(nb - 8)
    flags = torch.zeros(p.N + 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(rlqr.RlqrError, match="workspace"):
        rlqr.rlqr_factor(dp, opts, small, flags)
    big = rlqr.alloc_workspace(nb + 512)
    with pytest.raises(rlqr.RlqrError, match="workspace"):
        rlqr.rlqr_factor(dp, opts, big[8:], flags)  # misaligned


def _batch_parity(batch_host, dbatch, prec, out):
    st, xo, uo, yo, fo = oracle.riccati_batch(batch_host)
    rels = []
    for b in range(batch_host.count):
        x, u, y, f = dbatch.instance_view(b)
        np.testing.assert_array_equal(f, fo[b])
        p = batch_host.instance(b)
        rel = oracle.residual(p, x, u, y).rel
        rels.append(rel)
        want = rlqr.RLQR_NOT_PD if st[b] == oracle.NOT_PD else rlqr.RLQR_OK
        assert out["status"][b] == want
    rels = np.array(rels)
    assert rels.max() <= REL_TOL, f"max oracle rel-resid {rels.max():.3e}"
    if out["rel"] is not None:
        # the device's residual bookkeeping agrees with the oracle's
        assert np.all(out["rel"] <= REL_TOL)
        if prec == rlqr.RLQR_FP64:
            # the FP64 path reports the residual itself: equal up to rounding
            np.testing.assert_allclose(out["rel"], rels, rtol=0.05, atol=2e-14)
        else:
            # the mixed path reports an upper bound: its updated residual plus
            # the accumulated rounding bound of the FP32 products of the
            # corrections, so that a certified convergence never rests on
            # an underestimate
            assert np.all(rels <= 1.05 * out["rel"] + 1e-15), \
                np.max(rels / np.maximum(out["rel"], 1e-300))
    return rels


@pytest.mark.parametrize("prec", PRECS)
def test_workload2_small_batch(prec):
    """64 instances, N=64, n=12, m=4 (30% non-convex, 5% pivot-indefinite)."""
    bh = inputs.workload2(count=64, N=64)
    db = rlqr.DeviceBatch.from_uniform(bh)
    out = solve_batch(db, prec)
    _batch_parity(bh, db, prec, out)


@pytest.mark.parametrize("prec", PRECS)
def test_batched_solve_is_bitwise_deterministic(prec):
    """Two solves of the same batch (fresh workspaces, the outputs cleared in
    between): x, u, y, the pivot flags, the backward errors, statuses and
    refinement counts are bit-identical -- no reduction order or race
    depends on scheduling."""
    bh = inputs.workload2(count=148, N=64)
    db = rlqr.DeviceBatch.from_uniform(bh)
    runs = []
    for _ in range(2):
        for t in (db.x, db.u, db.y):
            t.fill_(float("nan"))
        db.pivot_pd.fill_(0xAB)
        out = solve_batch(db, prec)
        runs.append(dict(x=db.x.clone(), u=db.u.clone(), y=db.y.clone(),
                         f=db.pivot_pd.clone(), rel=out["rel"], st=out["status"], it=out["iters"]))
    a, b = runs
    for k in ("x", "u", "y", "f"):
        assert torch.equal(a[k].view(torch.uint8), b[k].view(torch.uint8)), k
    for k in ("rel", "st", "it"):
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k


@pytest.mark.parametrize("prec", PRECS)
def test_workload2_full_batch(prec):
    """The full 1024-instance workload (n=12, m=4, N=256), every instance
    checked: flags byte-identical, oracle rel-resid <= 1e-9."""
    bh = inputs.workload2()
    db = rlqr.DeviceBatch.from_uniform(bh)
    out = solve_batch(db, prec)
    rels = _batch_parity(bh, db, prec, out)
    if prec == rlqr.RLQR_MIXED:
        assert out["iters"].max() <= 3


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_batch(prec):
    """Instances of different (N, n, m) in one call, including tails of
    every kernel bucket."""
    dims = [(5, 3, 1), (64, 12, 4), (1, 1, 1), (33, 6, 2), (17, 24, 8), (9, 48, 16),
            (100, 4, 2), (2, 16, 5)]
    probs = [inputs.random_instance(200 + i, N, n, m, 10.0 ** (-1 - i % 6))
             for i, (N, n, m) in enumerate(dims)]
    db = rlqr.DeviceBatch.from_problems(probs)
    out = solve_batch(db, prec)
    for b, p in enumerate(probs):
        x, u, y, f = db.instance_view(b)
        ref = oracle.riccati(p)
        np.testing.assert_array_equal(f, ref.flags)
        assert oracle.residual(p, x, u, y).rel <= REL_TOL
        assert oracle.forward_error((ref.x, ref.u, ref.y), x, u, y) <= FWD_TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_workload4_sample(prec):
    """A sample shaped like the ragged workload (n in {6, 12, 24, 48},
    m = n/3, M != 0, barrier-scaled diagonals of Q and R, delta log-uniform)
    with horizons capped at 160: one call, instances grouped by size class
    and ordered longest first on the device; every instance checked against
    the oracle."""
    dims = inputs.workload4_dims(4096)[:40]
    probs = [inputs.workload4_instance(b, min(N, 160), n, m) for b, (N, n, m) in enumerate(dims)]
    db = rlqr.DeviceBatch.from_problems(probs)
    out = solve_batch(db, prec, max_refine=6)
    assert set(out["status"].tolist()) <= {rlqr.RLQR_OK, rlqr.RLQR_NOT_PD}
    for b, p in enumerate(probs):
        x, u, y, f = db.instance_view(b)
        ref = oracle.riccati(p)
        np.testing.assert_array_equal(f, ref.flags)
        assert oracle.residual(p, x, u, y).rel <= REL_TOL


@pytest.mark.parametrize("prec,route", [(rlqr.RLQR_FP64, None), (rlqr.RLQR_MIXED, None),
                                        (rlqr.RLQR_MIXED, rlqr.SWEEP_ROUTE_PERSISTENT)])
def test_ragged_batch_graph_replay(prec, route):
    """A ragged batch runs its size classes on the library's own streams,
    forked from and joined back to the caller's stream, or (mixed, route 4)
    all its sweeps in one persistent launch: the call can be captured into a
    CUDA graph, and a replay reproduces the eager call's solution, flags,
    status and backward errors bit for bit."""
    dims = inputs.workload4_dims(4096)[:24]
    probs = [inputs.workload4_instance(b, min(N, 96), n, m) for b, (N, n, m) in enumerate(dims)]
    assert len({(p.n, p.m) for p in probs}) > 1
    db = rlqr.DeviceBatch.from_problems(probs)
    opts = rlqr.make_opts(prec, tol=1e-9, max_refine=6)
    if route is not None:
        rlqr.rlqr_tune_batched_set(db, opts, route)
    ws = rlqr.alloc_workspace(rlqr.rlqr_batched_workspace_bytes(db, opts))
    B = db.count
    st = torch.full((B,), -1, dtype=torch.int32, device="cuda")
    rel = torch.full((B,), -1.0, dtype=torch.float64, device="cuda")
    it = torch.full((B,), -1, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # eager call (also creates the class streams)
        rlqr.rlqr_solve_batched(db, opts, ws, st, rel, it)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = [t.clone() for t in (db.x, db.u, db.y, db.pivot_pd, st, rel, it)]
    for t in (db.x, db.u, db.y, rel):
        t.fill_(float("nan"))
    db.pivot_pd.fill_(0)
    st.fill_(-1)
    it.fill_(-1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rlqr.rlqr_solve_batched(db, opts, ws, st, rel, it)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, (db.x, db.u, db.y, db.pivot_pd, st, rel, it)):
        assert torch.equal(a, b)
    for b, p in enumerate(probs):
        x, u, y, f = db.instance_view(b)
        np.testing.assert_array_equal(f, oracle.riccati(p).flags)
        assert oracle.residual(p, x, u, y).rel <= REL_TOL
    if route is not None:
        rlqr.rlqr_tune_batched_set(db, opts, 0)


def test_ragged_persistent_sweep_matches_class_streams():
    """The persistent sweep (one launch, work items longest chain first)
    against the per-class launches on the same ragged batch with every
    covered size and ragged tails of the 8-instance warp items: the same
    flags and statuses, each solution within 1e-9 of the oracle's backward
    error bar, and the tuner choosing one of the two sweep routes."""
    dims = [(40 + 7 * b, (4, 6, 12, 24, 32, 48)[b % 6], 0) for b in range(29)]
    probs = []
    for b, (N, n, _) in enumerate(dims):
        m = {4: 2, 6: 2, 12: 4, 24: 8, 32: 8, 48: 16}[n]
        probs.append(inputs.random_instance(600 + b, N, n, m, 10.0 ** (-2 - b % 5)))
    db = rlqr.DeviceBatch.from_problems(probs)
    opts = rlqr.make_opts(rlqr.RLQR_MIXED, tol=1e-9, max_refine=6)
    outs = {}
    for route in (rlqr.SWEEP_ROUTE_STREAMS, rlqr.SWEEP_ROUTE_PERSISTENT):
        rlqr.rlqr_tune_batched_set(db, opts, route)
        out = solve_batch(db, rlqr.RLQR_MIXED, max_refine=6)
        outs[route] = (out, [tuple(t.copy() for t in db.instance_view(b)) for b in range(len(probs))])
        for b, p in enumerate(probs):
            x, u, y, f = db.instance_view(b)
            ref = oracle.riccati(p)
            np.testing.assert_array_equal(f, ref.flags, err_msg=f"route {route} instance {b}")
            assert oracle.residual(p, x, u, y).rel <= REL_TOL, (route, b)
    a, b_ = outs[rlqr.SWEEP_ROUTE_STREAMS][0], outs[rlqr.SWEEP_ROUTE_PERSISTENT][0]
    np.testing.assert_array_equal(a["status"], b_["status"])
    ws = rlqr.alloc_workspace(rlqr.rlqr_batched_workspace_bytes(db, opts))
    route, ms = rlqr.rlqr_autotune_batched(db, opts, ws)
    assert route in (rlqr.SWEEP_ROUTE_STREAMS, rlqr.SWEEP_ROUTE_PERSISTENT) and ms > 0
    rlqr.rlqr_tune_batched_set(db, opts, 0)
    # a route of the other kind, or a batch the persistent sweep does not cover
    with pytest.raises(rlqr.RlqrError):
        rlqr.rlqr_tune_batched_set(db, opts, rlqr.RES_ROUTE_GRID)
    odd = rlqr.DeviceBatch.from_problems(probs[:3] + [inputs.random_instance(7, 20, 6, 1, 1e-3)])
    with pytest.raises(rlqr.RlqrError):
        rlqr.rlqr_tune_batched_set(odd, opts, rlqr.SWEEP_ROUTE_PERSISTENT)


@pytest.mark.parametrize("dims", [(6, 1), (12, 4), (24, 8), (32, 8), (48, 16), (10, 3)],
                         ids=lambda d: f"n{d[0]}m{d[1]}")
@pytest.mark.parametrize("prec", PRECS)
def test_uniform_batch_every_residual_route(dims, prec):
    """Uniform batches at the sizes of every first-residual route (float-float
    warp residual, generic FP64 residual, stage-parallel grid residual) and
    of every sweep kernel; horizons differ inside the batch."""
    n, m = dims
    probs = [inputs.random_instance(300 + b, N, n, m, 10.0 ** (-2 - b))
             for b, N in enumerate((23, 7, 31))]
    db = rlqr.DeviceBatch.from_problems(probs)
    out = solve_batch(db, prec)
    assert set(out["status"].tolist()) <= {rlqr.RLQR_OK, rlqr.RLQR_NOT_PD}
    for b, p in enumerate(probs):
        x, u, y, f = db.instance_view(b)
        ref = oracle.riccati(p)
        np.testing.assert_array_equal(f, ref.flags)
        assert oracle.residual(p, x, u, y).rel <= REL_TOL
        assert out["rel"][b] <= 1e-9 or prec == rlqr.RLQR_FP64


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_workload4_full_horizons(prec):
    """The ragged bench's launch configuration at full size: the first 512
    instances of the ragged batch (N up to 2048, n up to 48, barrier-scaled
    diagonals) in one call.  Every instance's flags are byte-identical to the
    oracle's and its backward error on the GPU is <= 1e-9; per state
    dimension the longest instance and three others also have their solution
    checked by the oracle (rel-resid <= 1e-9)."""
    import multiprocessing as mp
    import os
    dims = inputs.workload4_dims(4096)[:512]
    items = list(enumerate(dims))
    with mp.get_context("spawn").Pool(min(32, os.cpu_count() or 1)) as pool:
        probs = pool.map(workload4_item, items, chunksize=4)
        ref_flags = pool.map(workload4_oracle_flags, items, chunksize=2)
    db = rlqr.DeviceBatch.from_problems(probs)
    out = solve_batch(db, prec, max_refine=6)
    assert set(out["status"].tolist()) <= {rlqr.RLQR_OK, rlqr.RLQR_NOT_PD}
    assert out["rel"].max() <= REL_TOL
    for b in range(len(dims)):
        _, _, _, f = db.instance_view(b)
        np.testing.assert_array_equal(f, ref_flags[b], err_msg=f"instance {b} {dims[b]}")
    for nx in (6, 12, 24, 48):
        idx = [b for b, d in enumerate(dims) if d[1] == nx]
        sample = sorted({max(idx, key=lambda b: dims[b][0])} | set(idx[:3]))
        for b in sample:
            x, u, y, f = db.instance_view(b)
            ref = oracle.riccati(probs[b])
            np.testing.assert_array_equal(f, ref.flags)
            assert oracle.residual(probs[b], x, u, y).rel <= REL_TOL
