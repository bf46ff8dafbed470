"""General diagonal dual regularization Delta_i = diag(d_i) on the GPU
(rlqr_solve_diag) against the oracle: pivot flags byte-identical to the
oracle's recursion with S_i = I + Delta_i^{1/2} P_i Delta_i^{1/2}, backward
error of the ORIGINAL system (dense, assembled by the oracle) <= 1e-9, the
forward error to the dense solution, both precisions, SEQ and SCAN, an
indefinite case, a non-positive d_i, and RLQR_OPT_SYNC."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_16370_b300 import inputs, rlqr

pytestmark = pytest.mark.gpu


def _run(prob, d, prec, algo=rlqr.RLQR_ALGO_SEQ, sync=False):
    N, n, m = prob.N, prob.n, prob.m
    dp = rlqr.DeviceProblem.from_host(prob)
    opts = rlqr.make_opts(prec, algo=algo, tol=1e-9, max_refine=4, sync=sync)
    ws = rlqr.alloc_workspace(rlqr.rlqr_diag_workspace_bytes(N, n, m, opts))
    f = dict(dtype=torch.float64, device="cuda")
    x, u, y = torch.zeros(N + 1, n, **f), torch.zeros(N, m, **f), torch.zeros(N + 1, n, **f)
    flags = torch.zeros(N + 1, dtype=torch.uint8, device="cuda")
    rel = torch.full((1,), -1.0, **f)
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    code = rlqr.rlqr_solve_diag(dp, torch.from_numpy(np.ascontiguousarray(d)).cuda(), opts, ws,
                                x, u, y, flags, rel, st)
    torch.cuda.synchronize()
    return dict(code=code, status=int(st.item()), rel=float(rel.item()), x=x.cpu().numpy(),
                u=u.cpu().numpy(), y=y.cpu().numpy(), flags=flags.cpu().numpy())


def _backward_error(prob, d, x, u, y):
    K, b = oracle.kkt_dense_diag(prob, d)
    z = oracle.join_solution(prob, x, u, y)
    r = K @ z + b
    return np.abs(r).max() / (np.abs(K).sum(axis=1).max() * np.abs(z).max() + np.abs(b).max())


CASES = [(61, 40, 4, 2, -5, -1, rlqr.RLQR_ALGO_SEQ), (62, 33, 12, 4, -6, -2, rlqr.RLQR_ALGO_SEQ),
         (63, 64, 6, 2, -4, -1, rlqr.RLQR_ALGO_SCAN), (64, 20, 24, 8, -5, -2, rlqr.RLQR_ALGO_SEQ),
         (65, 48, 12, 4, -8, 0, rlqr.RLQR_ALGO_SCAN)]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[1]}n{c[2]}a{c[6]}" for c in CASES])
@pytest.mark.parametrize("prec", [rlqr.RLQR_FP64, rlqr.RLQR_MIXED])
def test_diag_delta_matches_the_oracle(case, prec):
    seed, N, n, m, lo, hi, algo = case
    prob = inputs.random_instance(seed, N, n, m, 1e-3)
    d = 10.0 ** np.random.default_rng(seed).uniform(lo, hi, (N + 1, n))
    out = _run(prob, d, prec, algo)
    assert out["code"] == rlqr.RLQR_OK and out["status"] in (rlqr.RLQR_OK, rlqr.RLQR_NOT_PD)
    x, u, y, flags = oracle.riccati_diag(prob, d)
    np.testing.assert_array_equal(out["flags"], flags)
    be = _backward_error(prob, d, out["x"], out["u"], out["y"])
    assert be <= 1e-9
    # the library's own FP64 residual of the original system reports it
    assert abs(out["rel"] - be) <= 0.1 * be + 1e-16
    K, b = oracle.kkt_dense_diag(prob, d)
    zr = np.linalg.solve(K, -b)
    z = oracle.join_solution(prob, out["x"], out["u"], out["y"])
    tol = 1e-8 if prec == rlqr.RLQR_FP64 else 1e-6
    assert np.abs(z - zr).max() <= tol * max(1.0, np.abs(zr).max())


@pytest.mark.parametrize("prec", [rlqr.RLQR_FP64, rlqr.RLQR_MIXED])
def test_indefinite_and_degenerate_cases(prec):
    prob = inputs.random_instance(70, 24, 4, 2, 1e-3)
    Q = prob.Q.copy()
    Q -= 3.0 * np.eye(4)
    prob.Q = Q
    d = 10.0 ** np.random.default_rng(70).uniform(-3, 1, (25, 4))
    out = _run(prob, d, prec)
    x, u, y, flags = oracle.riccati_diag(prob, d)
    np.testing.assert_array_equal(out["flags"], flags)
    assert not np.all(flags == 3)
    assert out["status"] == rlqr.RLQR_NOT_PD
    assert _backward_error(prob, d, out["x"], out["u"], out["y"]) <= 1e-9
    # a zero entry of Delta: non-finite scaled data, reported (synchronously
    # with RLQR_OPT_SYNC) as a singular pivot
    d0 = d.copy()
    d0[5, 2] = 0.0
    bad = _run(inputs.random_instance(71, 24, 4, 2, 1e-3), d0, prec, sync=True)
    assert bad["code"] == rlqr.RLQR_ERR_SINGULAR and bad["status"] == rlqr.RLQR_ERR_SINGULAR
