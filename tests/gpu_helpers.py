"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare with the FP64 oracle on the same seeded inputs.

Parity bar (floating point): the oracle's FP64 residual of the GPU solution
must have normwise backward error ||Kz+b|| / (||K|| ||z|| + ||b||) <= 1e-9,
and the per-stage pivot-PD flags must be byte-identical to the oracle's.
As a secondary check the forward error to the oracle's solution is bounded
(FP64 path 1e-8, mixed path 1e-6 on the test instances; both far above the
observed values and derived from rel <= 1e-9 times the modest condition of
these instances)."""
import numpy as np
import torch

import oracle
from paper_2509_16370_b300 import rlqr

REL_TOL = 1e-9
FWD_TOL = {rlqr.RLQR_FP64: 1e-8, rlqr.RLQR_MIXED: 1e-6}


def solve_single(p, prec, max_refine=3, factor_only=False, tol=1e-9, algo=rlqr.RLQR_ALGO_AUTO):
    dp = rlqr.DeviceProblem.from_host(p)
    opts = rlqr.make_opts(prec, algo=algo, tol=tol, max_refine=max_refine)
    nb = rlqr.rlqr_workspace_bytes(p.N, p.n, p.m, opts)
    ws = rlqr.alloc_workspace(nb)
    flags = torch.zeros(p.N + 1, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rlqr.rlqr_factor(dp, opts, ws, flags, status)
    x = torch.zeros(p.N + 1, p.n, dtype=torch.float64, device="cuda")
    u = torch.zeros(p.N, p.m, dtype=torch.float64, device="cuda")
    y = torch.zeros(p.N + 1, p.n, dtype=torch.float64, device="cuda")
    rel = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    iters = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st2 = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rlqr.rlqr_solve(dp, opts, ws, x, u, y, rel, iters, st2)
    torch.cuda.synchronize()
    return dict(x=x.cpu().numpy(), u=u.cpu().numpy(), y=y.cpu().numpy(),
                flags=flags.cpu().numpy(), status_factor=int(status.item()),
                status=int(st2.item()), rel=float(rel.item()), iters=int(iters.item()),
                dp=dp, ws=ws, opts=opts)


def check_against_oracle(p, out, prec, rel_tol=REL_TOL):
    ref = oracle.riccati(p)
    assert ref.status in (oracle.OK, oracle.NOT_PD)
    np.testing.assert_array_equal(out["flags"], ref.flags)
    res = oracle.residual(p, out["x"], out["u"], out["y"])
    assert res.rel <= rel_tol, f"oracle rel-resid of GPU solution {res.rel:.3e}"
    fe = oracle.forward_error((ref.x, ref.u, ref.y), out["x"], out["u"], out["y"])
    assert fe <= FWD_TOL[prec], f"forward error {fe:.3e}"
    return res.rel, fe, ref


def solve_batch(dbatch, prec, max_refine=3, want_rel=True, tol=1e-9):
    opts = rlqr.make_opts(prec, tol=tol, max_refine=max_refine)
    nb = rlqr.rlqr_batched_workspace_bytes(dbatch, opts)
    ws = rlqr.alloc_workspace(nb)
    B = dbatch.count
    status = torch.full((B,), -1, dtype=torch.int32, device="cuda")
    rel = torch.full((B,), -1.0, dtype=torch.float64, device="cuda") if want_rel else None
    iters = torch.full((B,), -1, dtype=torch.int32, device="cuda")
    rlqr.rlqr_solve_batched(dbatch, opts, ws, status, rel, iters)
    torch.cuda.synchronize()
    return dict(status=status.cpu().numpy(), rel=None if rel is None else rel.cpu().numpy(),
                iters=iters.cpu().numpy(), ws=ws)


def workload4_item(arg):
    """Instance b of the ragged workload with its (N, n, m) (a worker of a
    spawn process pool)."""
    from paper_2509_16370_b300 import inputs
    b, (N, n, m) = arg
    return inputs.workload4_instance(b, N, n, m)


def workload4_oracle_flags(arg):
    """The oracle's pivot flags of instance b of the ragged workload (a worker
    of a spawn process pool: it regenerates the instance from its seed)."""
    import oracle
    return oracle.riccati(workload4_item(arg)).flags
