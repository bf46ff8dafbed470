"""GPU test of the allocation-free entry point rlqr_solve_noalloc.

Callers such as a control loop that may not allocate device memory after
start-up (or code inside another runtime that owns the allocator) cannot call
cudaMalloc; rlqr_solve_noalloc gives them the solve with the library's own
static device scratch.  This file is collected last on purpose: if it fails,
a run that stops at the first failure has already run every other test.
It must also pass alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_16370_b300 import inputs
from paper_2509_16370_b300 import rlqr
from tests.gpu_helpers import FWD_TOL, REL_TOL, solve_single

pytestmark = pytest.mark.gpu


def _noalloc(p, prec):
    dp = rlqr.DeviceProblem.from_host(p)
    opts = rlqr.make_opts(prec, tol=1e-9, max_refine=3)
    x = torch.full((p.N + 1, p.n), np.nan, dtype=torch.float64, device="cuda")
    u = torch.full((p.N, p.m), np.nan, dtype=torch.float64, device="cuda")
    y = torch.full((p.N + 1, p.n), np.nan, dtype=torch.float64, device="cuda")
    flags = torch.zeros(p.N + 1, dtype=torch.uint8, device="cuda")
    rel = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rlqr.rlqr_solve_noalloc(dp, opts, x, u, y, flags, rel, st)
    torch.cuda.synchronize()
    return dict(x=x.cpu().numpy(), u=u.cpu().numpy(), y=y.cpu().numpy(),
                flags=flags.cpu().numpy(), rel=float(rel.item()), status=int(st.item()))


@pytest.mark.parametrize("prec", [rlqr.RLQR_FP64, rlqr.RLQR_MIXED])
def test_noalloc_matches_workspace_entry_points_twice(prec):
    """Two calls in a row (the second reuses the static scratch left by the
    first, on a different instance) agree with rlqr_factor + rlqr_solve on a
    caller-allocated workspace: identical flags and status, solutions equal
    within the parity tolerances, oracle rel-resid <= 1e-9."""
    probs = [inputs.workload1(), inputs.random_instance(301, 40, 12, 4, 3e-3, with_M=True)]
    probs[1].Q[5] -= 2.0 * np.eye(12)  # a non-convex stage as well
    for p in probs + probs[:1]:
        ref = solve_single(p, prec)
        out = _noalloc(p, prec)
        np.testing.assert_array_equal(out["flags"], ref["flags"])
        assert out["status"] == ref["status"]
        fe = oracle.forward_error((ref["x"], ref["u"], ref["y"]), out["x"], out["u"], out["y"])
        assert fe <= FWD_TOL[prec]
        assert oracle.residual(p, out["x"], out["u"], out["y"]).rel <= REL_TOL
        assert out["rel"] <= REL_TOL


@pytest.mark.parametrize("dims", [(40, 24, 8), (128, 6, 1), (30, 10, 3), (20, 12, 3)],
                         ids=["cta_24x8", "tableau_6x1", "bucket_10x3", "tableau_12x3"])
@pytest.mark.parametrize("prec", [rlqr.RLQR_FP64, rlqr.RLQR_MIXED])
def test_noalloc_other_kernel_routes(dims, prec):
    """The sizes whose sweeps take the other routes -- the compile-time CTA
    sweep with its deferred certificate (24, 8), the tableau warp sweep with
    odd n_u (6, 1) and (12, 3), the bucket kernels at a size without an
    instantiation (10, 3) -- give the same flags, status and (within the
    parity tolerance) solution as rlqr_factor + rlqr_solve."""
    N, n, m = dims
    p = inputs.random_instance(400 + n, N, n, m, 1e-3, with_M=True)
    ref = solve_single(p, prec)
    out = _noalloc(p, prec)
    np.testing.assert_array_equal(out["flags"], ref["flags"])
    assert out["status"] == ref["status"]
    fe = oracle.forward_error((ref["x"], ref["u"], ref["y"]), out["x"], out["u"], out["y"])
    assert fe <= FWD_TOL[prec]
    assert oracle.residual(p, out["x"], out["u"], out["y"]).rel <= REL_TOL


def test_noalloc_refuses_the_scan():
    """The allocation-free call runs the sequential recursion only."""
    p = inputs.workload1()
    dp = rlqr.DeviceProblem.from_host(p)
    opts = rlqr.make_opts(rlqr.RLQR_FP64, algo=rlqr.RLQR_ALGO_SCAN)
    t = torch.zeros((p.N + 1) * p.n, dtype=torch.float64, device="cuda")
    f = torch.zeros(p.N + 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(rlqr.RlqrError, match="argument"):
        rlqr.rlqr_solve_noalloc(dp, opts, t, t, t, f)


def test_noalloc_rejects_oversized_instances():
    """An instance whose workspace exceeds the static scratch is refused on
    the host with RLQR_ERR_WORKSPACE; nothing runs on the GPU."""
    opts = rlqr.make_opts(rlqr.RLQR_FP64)
    N, n, m = 4000, 48, 16
    assert rlqr.rlqr_workspace_bytes(N, n, m, opts) > rlqr.NOALLOC_SCRATCH_BYTES
    p = inputs.Problem(N, n, m, Q=np.zeros((1,)), M=np.zeros((1,)), R=np.zeros((1,)),
                       q=np.zeros((1,)), r=np.zeros((1,)), A=np.zeros((1,)), B=np.zeros((1,)),
                       c=np.zeros((1,)), delta=0.1)
    dp = rlqr.DeviceProblem.from_host(p)  # tiny placeholder buffers: never read
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(rlqr.RlqrError, match="workspace"):
        rlqr.rlqr_solve_noalloc(dp, opts, t, t, t, f)
