"""Pivot certificate near its decision boundary (Section "Inertia
Certification", Theorem riccati-inertia-certification-theorem): flags
byte-identical to the FP64 oracle when one pivot sits at a relative margin of
1e-3, 1e-5 or 1e-7, in both precisions, single instance and batch.

The cases come from tests/golden/margin_cases.json (written by
make_margin_cases.py with the oracle only).  The mixed path keeps an FP32
certificate decision only when it holds with the margin tau = 2^-15 of the
Jacobi-scaled pivot matrix and otherwise lets the FP64 recursion decide the
instance's flags (the instance is then marked as escalated in its state at
the start of the workspace: int32 at byte 56)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2509_16370_b300 import inputs, rlqr
from tests.gpu_helpers import REL_TOL, solve_batch, solve_single

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "margin_cases.json")
with open(GOLDEN) as _f:
    CASES = json.load(_f)["cases"]
ESCALATED_BYTE = 56  # InstState: 5 doubles, then pivot_status, iters, converged, r_singular, escalated


def case_problem(c):
    p = inputs.random_instance(c["seed"], c["N"], c["n"], c["m"], c["delta"])
    if c["kind"] == "G":
        p.R = p.R.copy()
        p.R[c["kstar"]] -= c["alpha"] * np.eye(c["m"])
    else:
        p.Q = p.Q.copy()
        p.Q[c["kstar"]] -= c["alpha"] * np.eye(c["n"])
    return p


def escalated(ws):
    return int(ws[ESCALATED_BYTE:ESCALATED_BYTE + 4].cpu().numpy().view(np.int32)[0])


TAU = 2.0 ** -15


def check_escalation(case, esc):
    """The margin is stated for the Jacobi-scaled pivot (scaled_margin: its
    smallest eigenvalue, from the oracle).  The FP32-computed pivot differs
    from the exact one by far less than tau/4 in that scaling on these
    instances, so a pivot within tau/4 of singular cannot be decided in
    FP32, an FP32 decision implies a scaled margin above tau/2, and a pivot
    at relative margin 1e-3 (scaled margin > 64 tau) needs no escalation."""
    lam = abs(case["scaled_margin"])
    if lam < TAU / 4:
        assert esc == 1, f"scaled margin {lam:.2e} must be decided in FP64"
    if esc == 0:
        assert lam > TAU / 2, f"decided in FP32 at scaled margin {lam:.2e}"
    if case["mu"] >= 1e-3:
        assert lam > 64 * TAU and esc == 0, "a clear pivot is decided by the FP32 certificate"


IDS = [f"{c['kind']}{'+' if c['sign'] > 0 else '-'}{c['mu']:.0e}_n{c['n']}" for c in CASES]


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("prec", [rlqr.RLQR_FP64, rlqr.RLQR_MIXED])
def test_margin_flags_single(case, prec):
    p = case_problem(case)
    ref = oracle.riccati(p)
    assert ref.status in (oracle.OK, oracle.NOT_PD)
    assert ref.flags[case["kstar"]] == case["oracle_flags_at_kstar"]
    out = solve_single(p, prec, max_refine=8)
    np.testing.assert_array_equal(out["flags"], ref.flags)
    want = rlqr.RLQR_OK if (ref.flags == 3).all() else rlqr.RLQR_NOT_PD
    assert out["status_factor"] == want
    rel = oracle.residual(p, out["x"], out["u"], out["y"]).rel
    if prec == rlqr.RLQR_MIXED and case["mu"] <= 1e-7:
        # a pivot at relative margin 1e-7 makes kappa(K) u_32 ~ 1: refinement
        # with the FP32 factor contracts slowly; the call must not claim a
        # convergence the oracle does not confirm
        assert rel <= REL_TOL or out["status"] == rlqr.RLQR_ERR_NOT_CONVERGED, \
            (rel, out["rel"], out["iters"], out["status"])
        assert rel <= 1e-8
    else:
        assert rel <= REL_TOL
    if prec == rlqr.RLQR_MIXED:
        check_escalation(case, escalated(out["ws"]))


@pytest.mark.parametrize("prec", [rlqr.RLQR_FP64, rlqr.RLQR_MIXED])
def test_margin_flags_batch(prec):
    """All cases in one ragged batch: escalated and decided instances side by
    side, every instance's flags equal to the oracle's."""
    probs = [case_problem(c) for c in CASES]
    db = rlqr.DeviceBatch.from_problems(probs)
    out = solve_batch(db, prec, max_refine=8)
    for b, p in enumerate(probs):
        x, u, y, f = db.instance_view(b)
        ref = oracle.riccati(p)
        np.testing.assert_array_equal(f, ref.flags, err_msg=IDS[b])
        want = rlqr.RLQR_OK if (ref.flags == 3).all() else rlqr.RLQR_NOT_PD
        rel = oracle.residual(p, x, u, y).rel
        if prec == rlqr.RLQR_MIXED and CASES[b]["mu"] <= 1e-7:
            assert (rel <= REL_TOL and out["status"][b] == want) or \
                out["status"][b] == rlqr.RLQR_ERR_NOT_CONVERGED, IDS[b]
            assert rel <= 1e-8, IDS[b]
        else:
            assert out["status"][b] == want, IDS[b]
            assert rel <= REL_TOL, IDS[b]
