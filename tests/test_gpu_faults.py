"""Faulty inputs on every GPU path: the library reports them through the
per-instance status and keeps the other instances of a batch intact (no
trap, no hang: every decision is a host-visible status).

* a NaN or an infinity in the data makes a pivot non-finite: RLQR_ERR_SINGULAR
  (uniform batch, ragged batch, single instance on the sequential and on the
  associative-scan path, both precisions);
* a singular R_i is fine for the sequential recursion (it only needs G_i
  invertible) but the scan eliminates the controls through R_i^{-1}: there it
  is RLQR_ERR_SINGULAR, while the sequential path still matches the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_16370_b300 import inputs, rlqr
from tests.gpu_helpers import REL_TOL, solve_batch, solve_single

pytestmark = pytest.mark.gpu

PRECS = [rlqr.RLQR_FP64, rlqr.RLQR_MIXED]


def _poison(p, field, stage, value):
    arr = getattr(p, field).copy()
    arr[stage].flat[0] = value
    setattr(p, field, arr)
    return p


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("field,value", [("Q", np.nan), ("B", np.inf), ("A", -np.inf)])
def test_bad_data_in_batches(prec, field, value):
    """Uniform batch (warp kernels) and ragged batch (CTA sweep, grid
    residual): the poisoned instance reports RLQR_ERR_SINGULAR, the others
    are solved to the tolerance."""
    uni = [inputs.random_instance(600 + b, 40, 12, 4, 1e-3) for b in range(4)]
    rag = [inputs.workload4_instance(b, 30 + 5 * b, n, n // 3)
           for b, n in enumerate((6, 24, 48, 12))]
    for probs in (uni, rag):
        bad = 1
        probs[bad] = _poison(probs[bad], field, 7, value)
        db = rlqr.DeviceBatch.from_problems(probs)
        out = solve_batch(db, prec, max_refine=6)
        assert out["status"][bad] == rlqr.RLQR_ERR_SINGULAR
        for b, p in enumerate(probs):
            if b == bad:
                continue
            assert out["status"][b] in (rlqr.RLQR_OK, rlqr.RLQR_NOT_PD)
            x, u, y, f = db.instance_view(b)
            assert oracle.residual(p, x, u, y).rel <= REL_TOL


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("algo", [rlqr.RLQR_ALGO_SEQ, rlqr.RLQR_ALGO_SCAN])
def test_bad_data_single_instance(prec, algo):
    p = _poison(inputs.random_instance(610, 64, 4, 2, 1e-3), "Q", 20, np.nan)
    out = solve_single(p, prec, algo=algo)
    assert out["status_factor"] == rlqr.RLQR_ERR_SINGULAR
    assert out["status"] == rlqr.RLQR_ERR_SINGULAR


@pytest.mark.parametrize("prec", PRECS)
def test_singular_R_scan_reports_sequential_solves(prec):
    p = inputs.random_instance(611, 64, 4, 2, 1e-3)
    R = p.R.copy()
    R[30] = 0.0           # G_30 = B^T W B stays PD (B has full column rank)
    p.R = R
    seq = solve_single(p, prec, algo=rlqr.RLQR_ALGO_SEQ)
    ref = oracle.riccati(p)
    assert seq["status"] in (rlqr.RLQR_OK, rlqr.RLQR_NOT_PD)
    np.testing.assert_array_equal(seq["flags"], ref.flags)
    assert oracle.residual(p, seq["x"], seq["u"], seq["y"]).rel <= REL_TOL
    scan = solve_single(p, prec, algo=rlqr.RLQR_ALGO_SCAN)
    assert scan["status_factor"] == rlqr.RLQR_ERR_SINGULAR
    assert scan["status"] == rlqr.RLQR_ERR_SINGULAR
    # a later factorization of a regular instance in the same workspace shape
    # starts with a clear record
    ok = solve_single(inputs.random_instance(612, 64, 4, 2, 1e-3), prec,
                      algo=rlqr.RLQR_ALGO_SCAN)
    assert ok["status"] in (rlqr.RLQR_OK, rlqr.RLQR_NOT_PD)


@pytest.mark.parametrize("prec", PRECS)
def test_sync_option_returns_the_instance_status(prec):
    """RLQR_OPT_SYNC: the single-instance calls wait for their stream and
    return the instance status (here RLQR_ERR_SINGULAR for a NaN in the data,
    RLQR_OK / RLQR_NOT_PD for a regular instance); without it the host return
    stays RLQR_OK and the status is only on the device."""
    for p, bad in ((inputs.random_instance(620, 40, 4, 2, 1e-3), False),
                   (_poison(inputs.random_instance(621, 40, 4, 2, 1e-3), "Q", 9, np.nan), True)):
        dp = rlqr.DeviceProblem.from_host(p)
        for sync in (False, True):
            opts = rlqr.make_opts(prec, sync=sync)
            ws = rlqr.alloc_workspace(rlqr.rlqr_workspace_bytes(p.N, p.n, p.m, opts))
            flags = torch.zeros(p.N + 1, dtype=torch.uint8, device="cuda")
            x = torch.zeros(p.N + 1, p.n, dtype=torch.float64, device="cuda")
            u = torch.zeros(p.N, p.m, dtype=torch.float64, device="cuda")
            y = torch.zeros(p.N + 1, p.n, dtype=torch.float64, device="cuda")
            rel = torch.zeros(1, dtype=torch.float64, device="cuda")
            cf = rlqr.rlqr_factor(dp, opts, ws, flags)
            cs = rlqr.rlqr_solve(dp, opts, ws, x, u, y, rel)
            cn = rlqr.rlqr_solve_noalloc(dp, opts, x, u, y, flags, rel)
            torch.cuda.synchronize()
            if not sync:
                assert (cf, cs, cn) == (rlqr.RLQR_OK,) * 3
            elif bad:
                assert (cf, cs, cn) == (rlqr.RLQR_ERR_SINGULAR,) * 3
            else:
                assert cf in (rlqr.RLQR_OK, rlqr.RLQR_NOT_PD) and cs == cn == cf
