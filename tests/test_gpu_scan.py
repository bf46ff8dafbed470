"""GPU parity of the associative-scan path (Section "Parallel Algorithm"):
interval elements, chunked reverse scan with the combination rule, per-chunk
finalize, p-recurrence and composed affine x maps, then (mixed precision)
FP64 residual and refinement.

Bar (as for the sequential path): byte-identical pivot flags, the oracle's
FP64 normwise backward error of the GPU solution <= 1e-9, forward error to
the oracle's solution within the tolerances of gpu_helpers.  The chunk
length for these horizons is 8 stages, so N = 64 .. 203 spans 8 .. 26
chunks, several scan levels and a ragged last chunk; N = 5 is one partial
chunk.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_16370_b300 import inputs
from paper_2509_16370_b300 import rlqr
from tests.gpu_helpers import FWD_TOL, REL_TOL, check_against_oracle, solve_single

pytestmark = pytest.mark.gpu

SCAN = rlqr.RLQR_ALGO_SCAN
PRECS = [rlqr.RLQR_FP64, rlqr.RLQR_MIXED]


def _case(seed, N, n, m, delta, nonconvex=False):
    p = inputs.random_instance(seed, N, n, m, delta, with_M=True)
    if nonconvex:
        p.Q[N // 2] -= 3.0 * np.eye(n)
        p.Q[N // 3, 0, 0] -= 2.0
    return p


CASES = [
    ("n4m2_N64", lambda: inputs.workload1()),
    ("n4m2_N203", lambda: _case(401, 203, 4, 2, 1e-3)),
    ("n6m2_N150", lambda: _case(402, 150, 6, 2, 0.05)),
    ("n12m4_N131", lambda: _case(403, 131, 12, 4, 1e-4)),
    ("n12m4_N5", lambda: _case(404, 5, 12, 4, 0.2)),
    ("n32m8_N97", lambda: _case(405, 97, 32, 8, 1e-5)),
    ("n12m4_N120_nonconvex", lambda: _case(406, 120, 12, 4, 0.01, nonconvex=True)),
    # chunks of 21 stages: the P-only pass starts from the inner elements
    # (a final chunk of 12 stages without one)
    ("n12m4_N9000", lambda: _case(408, 9000, 12, 4, 1e-3)),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_scan_matches_oracle(name, make, prec):
    p = make()
    out = solve_single(p, prec, algo=SCAN)
    assert out["status"] in (rlqr.RLQR_OK, rlqr.RLQR_NOT_PD), out["status"]
    rel, fe, ref = check_against_oracle(p, out, prec)
    assert out["status_factor"] == ref.status
    if prec == rlqr.RLQR_MIXED:
        # the reported value bounds the backward error from above (updated
        # residual plus the accumulated rounding bound of the corrections)
        assert out["rel"] <= REL_TOL
        assert rel <= 1.05 * out["rel"] + 1e-15, (rel, out["rel"])


@pytest.mark.parametrize("prec", PRECS)
def test_scan_agrees_with_sequential(prec):
    p = _case(407, 173, 12, 4, 3e-3)
    a = solve_single(p, prec, algo=SCAN)
    b = solve_single(p, prec, algo=rlqr.RLQR_ALGO_SEQ)
    np.testing.assert_array_equal(a["flags"], b["flags"])
    fe = oracle.forward_error((b["x"], b["u"], b["y"]), a["x"], a["u"], a["y"])
    assert fe <= FWD_TOL[prec]


def test_auto_selects_by_horizon():
    """AUTO runs the sequential recursion for short horizons and the scan from
    N = 4096 on (same results as the explicit choice)."""
    short = _case(408, 40, 4, 2, 0.01)
    a = solve_single(short, rlqr.RLQR_FP64)
    b = solve_single(short, rlqr.RLQR_FP64, algo=rlqr.RLQR_ALGO_SEQ)
    np.testing.assert_array_equal(a["x"], b["x"])
    long = _case(409, 4096, 4, 2, 0.01)
    a = solve_single(long, rlqr.RLQR_FP64)
    b = solve_single(long, rlqr.RLQR_FP64, algo=SCAN)
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["flags"], b["flags"])


def test_scan_rejects_what_it_does_not_cover():
    opts = rlqr.make_opts(rlqr.RLQR_FP64, algo=SCAN)
    for p in (_case(410, 20, 4, 2, 0.0), _case(411, 20, 5, 2, 0.1)):  # delta = 0; no kernel for (5,2)
        dp = rlqr.DeviceProblem.from_host(p)
        ws = rlqr.alloc_workspace(max(rlqr.rlqr_workspace_bytes(p.N, p.n, p.m, opts), 256))
        flags = torch.zeros(p.N + 1, dtype=torch.uint8, device="cuda")
        with pytest.raises(rlqr.RlqrError, match="argument"):
            rlqr.rlqr_factor(dp, opts, ws, flags)


@pytest.mark.parametrize("prec", PRECS)
def test_long_horizon_n32(prec):
    """The long-horizon workload's shape at a reduced horizon (n=32, m=8,
    N=4096, delta=1e-7, rho(A)=0.99, Q and R with condition number 1e4):
    512 chunks, ten scan levels."""
    p = inputs.workload3(N=4096)
    out = solve_single(p, prec, algo=SCAN)
    assert out["status"] in (rlqr.RLQR_OK, rlqr.RLQR_NOT_PD)
    check_against_oracle(p, out, prec)


def test_long_horizon_full_size_mixed():
    """The long-horizon workload at full size (n=32, m=8, N=65536, 444
    chunks): mixed-precision scan, one refinement pass, flags identical to
    the oracle's and the oracle's backward error of the solution <= 1e-9."""
    p = inputs.workload3()
    out = solve_single(p, rlqr.RLQR_MIXED, algo=SCAN)
    assert out["status"] in (rlqr.RLQR_OK, rlqr.RLQR_NOT_PD)
    assert out["rel"] <= REL_TOL
    check_against_oracle(p, out, rlqr.RLQR_MIXED)
