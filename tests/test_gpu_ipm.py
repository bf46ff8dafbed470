"""The batched regularized IPM on the GPU against the oracle's IPM (Section
"The Regularized Interior Point Method", Section "Applying the regularized
IPM to optimal control").

* linearization: the LQR data of the Newton system, the KKT error and the
  barrier update at the same point, element by element;
* one iteration at a time: from the GPU's state before an iteration, the
  oracle's iteration (inertia correction, line search, update) reproduces the
  GPU's state after it, on cold starts of the workload's swing-up instances
  (so chaotic growth of rounding differences over many iterations does not
  enter the comparison);
* whole solves on instances that converge: same status and iteration count,
  and the final point passes the oracle's own KKT error test;
* the full batch of 8192 instances: invariants of the iterates and the KKT
  error recomputed by the oracle on a sample.
"""
import numpy as np
import pytest
import torch

import oracle.ipm as O
from paper_2509_16370_b300 import inputs
from paper_2509_16370_b300 import ipm as G

pytestmark = pytest.mark.gpu

FP64 = dict(hessian=G.RLQR_IPM_HESS_EXACT_FP64, lqr_prec=G.RLQR_FP64)


def _setup(bs, N=128, **kw):
    x0 = np.stack([inputs.workload5_instance(b)[0] for b in bs])
    xg = np.stack([inputs.workload5_instance(b)[1] for b in bs])
    model = G.make_model(N=N)
    opts = G.make_ipm_opts(**{**FP64, **kw})
    st = G.IpmState(len(bs), N)
    ws = G.alloc_ipm_workspace(len(bs), model, opts)
    dx0, dxg = torch.from_numpy(x0).cuda(), torch.from_numpy(xg).cuda()
    G.rlqr_ipm_init(model, opts, dx0, st)
    return model, opts, st, ws, dx0, dxg, x0, xg


def _oracle_opts(opts):
    return O.Options(max_iter=opts.max_iter, tol=opts.tol, eta=opts.eta,
                     exact_hessian=opts.hessian != G.RLQR_IPM_HESS_GAUSS_NEWTON)


def _oracle_state(st, b, x0, xg):
    h = lambda t: t[b].cpu().numpy().copy()  # noqa: E731
    return O.State(x0[b].copy(), xg[b].copy(), h(st.X), h(st.U), h(st.Y), h(st.S), h(st.Z),
                   float(st.mu[b]), float(st.rho[b]), int(st.iters[b]),
                   int(st.factorizations[b]), int(st.status[b]))


def _rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


def test_initial_point_matches_the_oracle():
    model, opts, st, ws, _, _, x0, xg = _setup(range(4))
    md, op = O.Model(), _oracle_opts(opts)
    for b in range(4):
        ref = O.initial_state(md, op, x0[b], xg[b])
        got = _oracle_state(st, b, x0, xg)
        assert _rel(got.X, ref.X) <= 1e-12
        # S = max(-g, s_min) and Z = mu0 / S from the rolled-out cart position
        np.testing.assert_allclose(got.S, ref.S, rtol=1e-12)
        np.testing.assert_allclose(got.Z, ref.Z, rtol=1e-12)
        assert got.mu == ref.mu and got.iters == 0 and got.status == 0


@pytest.mark.parametrize("N", [1, 40, 300, 4096])
@pytest.mark.parametrize("hess", [G.RLQR_IPM_HESS_EXACT_FP64, G.RLQR_IPM_HESS_EXACT_FP32,
                                  G.RLQR_IPM_HESS_GAUSS_NEWTON])
def test_linearization_matches_the_oracle(hess, N):
    """Horizons of one stage, of a partial pass, of several passes of the
    128-thread CTA over the stages, and the largest the ABI accepts."""
    bs = [0, 3, 7]
    model, opts, st, ws, dx0, dxg, x0, xg = _setup(bs, N=N, hessian=hess)
    rng = np.random.default_rng(5)
    # a point away from the rollout: perturbed states, controls, duals
    st.X += 0.05 * torch.from_numpy(rng.standard_normal(tuple(st.X.shape))).cuda()
    st.U += torch.from_numpy(rng.standard_normal(tuple(st.U.shape))).cuda()
    st.Y += torch.from_numpy(rng.standard_normal(tuple(st.Y.shape))).cuda()
    md, op = O.Model(N=N), _oracle_opts(opts)
    before = [_oracle_state(st, i, x0, xg) for i in range(len(bs))]
    G.rlqr_ipm_linearize(model, opts, dx0, dxg, st, ws)
    v = G.rlqr_ipm_lqr_view(model, opts, st, ws)
    torch.cuda.synchronize()
    for i, s0 in enumerate(before):
        ref = s0.copy()
        lin = O.linearize(md, op, ref)
        assert abs(float(st.kkt[i]) - lin.err0) <= 1e-12 * max(1.0, lin.err0)
        if lin.err_mu <= op.kappa_mu * ref.mu:
            ref.mu = max(op.mu_min, min(0.2 * ref.mu, ref.mu ** 1.5))
        assert float(st.mu[i]) == pytest.approx(ref.mu, rel=1e-15)
        _, prob, *_ = O.newton_lqr(md, op, ref, lin, 0.0)
        for k in ("A", "B", "c", "q", "r"):
            got = v[k][i].cpu().numpy()
            assert _rel(got.reshape(getattr(prob, k).shape), getattr(prob, k)) <= 1e-12, k
        htol = 1e-4 if hess == G.RLQR_IPM_HESS_EXACT_FP32 else 1e-11
        for k in ("Q", "M", "R"):
            got = v[k][i].cpu().numpy()
            assert _rel(got.reshape(getattr(prob, k).shape), getattr(prob, k)) <= htol, k


@pytest.mark.parametrize("N", [128, 300])
def test_iterations_match_the_oracle_one_at_a_time(N):
    bs = [0, 1, 2, 5]
    model, opts, st, ws, dx0, dxg, x0, xg = _setup(bs, N=N)
    md, op = O.Model(N=N), _oracle_opts(opts)
    worst = 0.0
    for it in range(40):
        before = [_oracle_state(st, i, x0, xg) for i in range(len(bs))]
        G.rlqr_ipm_iterate(model, opts, dx0, dxg, st, ws)
        torch.cuda.synchronize()
        for i, s0 in enumerate(before):
            if s0.status != 0:
                continue
            ref = O.iterate(md, op, s0.copy())
            got = _oracle_state(st, i, x0, xg)
            assert (got.status, got.iters, got.factorizations) == \
                (ref.status, ref.iters, ref.factorizations), (it, i)
            assert got.rho == pytest.approx(ref.rho, rel=1e-12, abs=0.0)
            for k in ("X", "U", "S", "Y", "Z"):
                e = _rel(getattr(got, k), getattr(ref, k))
                worst = max(worst, e)
                assert e <= 1e-8, (it, i, k, e)
    assert worst <= 1e-8


def test_whole_solves_match_the_oracle():
    """Instances the oracle solves to the tolerance: the same outcome and
    iteration count, and the oracle's KKT error at the GPU's final point."""
    bs = [0, 5, 32]
    model, opts, st, ws, dx0, dxg, x0, xg = _setup(bs)
    n_it = G.rlqr_ipm_solve(model, opts, dx0, dxg, st, ws)
    torch.cuda.synchronize()
    md, op = O.Model(), _oracle_opts(opts)
    for i, b in enumerate(bs):
        ref = O.solve(md, op, x0[i], xg[i])
        got = _oracle_state(st, i, x0, xg)
        assert ref.status == 1
        assert got.status == G.CONVERGED
        assert abs(got.iters - ref.iters) <= 2
        assert O.kkt_error(md, op, got) <= op.tol
    assert n_it >= max(int(t) for t in st.iters.cpu())


def test_full_batch_invariants_and_sampled_kkt():
    """The 8192-instance batch with the FP32 Hessian and mixed-precision LQR
    solves, in the configuration the bench times: after a few iterations the
    slacks and bound duals stay positive and the iterates finite, and the KKT
    error the GPU computes at the current point equals the oracle's there
    (sampled instances)."""
    count = 8192
    x0, xg = inputs.workload5(count)
    model = G.make_model()
    opts = G.make_ipm_opts()
    st = G.IpmState(count, model.N)
    ws = G.alloc_ipm_workspace(count, model, opts)
    dx0, dxg = torch.from_numpy(x0).cuda(), torch.from_numpy(xg).cuda()
    G.rlqr_ipm_init(model, opts, dx0, st)
    for _ in range(5):
        G.rlqr_ipm_iterate(model, opts, dx0, dxg, st, ws)
    torch.cuda.synchronize()
    assert bool((st.S > 0).all()) and bool((st.Z >= 0).all())
    assert bool(torch.isfinite(st.X).all()) and bool(torch.isfinite(st.Y).all())
    assert set(st.status.unique().cpu().tolist()) <= {0, 1, 2, 3}
    assert int(st.iters.max()) == 5
    # the KKT error at the current point: a linearization of a copy
    probe = G.IpmState(count, model.N)
    for k in ("X", "U", "Y", "S", "Z", "mu", "rho", "iters", "factorizations", "status"):
        getattr(probe, k).copy_(getattr(st, k))
    G.rlqr_ipm_linearize(model, opts, dx0, dxg, probe, ws)
    torch.cuda.synchronize()
    md, op = O.Model(), _oracle_opts(opts)
    for b in np.random.default_rng(1).choice(count, 12, replace=False):
        if int(st.status[b]) != 0:
            continue
        lin = O.linearize(md, op, _oracle_state(st, b, x0, xg))
        assert abs(float(probe.kkt[b]) - lin.err0) <= 1e-10 * max(1.0, lin.err0)


def test_bench_configuration_matches_the_oracle_on_sampled_instances():
    """The configuration the bench times (8192 instances, FP32 Hessian term,
    mixed-precision LQR solves with FP64 refinement to 1e-9): for 16 sampled
    instances and each of 4 iterations, the oracle's iteration (FP64
    throughout) from the GPU's state before it gives the GPU's state after it.
    The FP32 Hessian term perturbs the Newton matrix by ~1e-7 relative, so the
    states agree to 1e-5 relative, except where that perturbation moves an
    Armijo test across its threshold (the accepted step then differs by a
    power of two): at most 2 such near-ties among the 64 comparisons."""
    count = 8192
    x0, xg = inputs.workload5(count)
    model = G.make_model()
    opts = G.make_ipm_opts()
    st = G.IpmState(count, model.N)
    ws = G.alloc_ipm_workspace(count, model, opts)
    dx0, dxg = torch.from_numpy(x0).cuda(), torch.from_numpy(xg).cuda()
    G.rlqr_ipm_init(model, opts, dx0, st)
    sample = np.random.default_rng(3).choice(count, 16, replace=False)
    md, op = O.Model(), _oracle_opts(opts)
    ties, compared = 0, 0
    for it in range(4):
        before = [_oracle_state(st, b, x0, xg) for b in sample]
        G.rlqr_ipm_iterate(model, opts, dx0, dxg, st, ws)
        torch.cuda.synchronize()
        for b, s0 in zip(sample, before):
            if s0.status != 0:
                continue
            ref = O.iterate(md, op, s0.copy())
            got = _oracle_state(st, b, x0, xg)
            compared += 1
            assert got.status == ref.status and got.iters == ref.iters
            e = max(_rel(getattr(got, k), getattr(ref, k)) for k in ("X", "U", "S", "Y", "Z"))
            if e > 1e-5:
                ties += 1
    assert compared >= 48
    assert ties <= 2, ties
