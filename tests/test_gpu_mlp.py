"""The warm-start network's CUDA kernels (BF16 tensor-core GEMMs with FP32
accumulation) against the FP64 oracle with BF16 rounding at the same points:
forward pass, loss and gradient, Adam step; and a short training run that
fits a teacher network.

Tolerances: the oracle accumulates in FP64 and the GPU in FP32, and a value
whose two sums straddle a BF16 rounding boundary rounds to neighbouring BF16
values (relative spacing 2^-8 = 3.9e-3) before the next layer, so the
comparisons are normwise at 2e-2 (forward) and 5e-2 (gradient blocks), far
below the size of the quantities, and exact for the Adam arithmetic up to
FP32 rounding."""
import numpy as np
import pytest
import torch

import oracle.mlp as M
from paper_2509_16370_b300 import mlp

pytestmark = pytest.mark.gpu


def _net(n_in, width, n_out, rows, seed):
    d = mlp.make_dims(n_in, width, n_out, rows)
    p = mlp.init_params(d, seed)
    rng = np.random.default_rng(seed)
    o, npad, total = M.layout(n_out, width)
    p[o["b1"][0]:o["b1"][0] + width] = rng.normal(size=width) * 0.1
    p[o["b3"][0]:o["b3"][0] + n_out] = rng.normal(size=n_out) * 0.1
    return d, p, mlp.WarmStartNet(d, p)


@pytest.mark.parametrize("dims", [(7, 64, 40, 32), (7, 256, 902, 64)])
def test_forward_and_gradient_match_the_oracle(dims):
    n_in, width, n_out, rows = dims
    d, p, net = _net(n_in, width, n_out, rows, 11)
    rng = np.random.default_rng(12)
    x = rng.normal(size=(rows * 2, n_in)).astype(np.float32)
    t = rng.normal(size=(rows * 2, n_out)).astype(np.float32)
    idx = rng.permutation(rows * 2)[:rows].astype(np.int32)
    y = net.forward(torch.from_numpy(x[:rows]).cuda()).cpu().numpy()
    yr, _ = M.forward(p.astype(np.float64), x[:rows].astype(np.float64), n_out, width)
    assert np.linalg.norm(y - yr) <= 2e-2 * np.linalg.norm(yr)
    loss, g = net.grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(),
                       torch.from_numpy(idx).cuda())
    lr_, gr = M.loss_and_grad(p.astype(np.float64), x[idx].astype(np.float64),
                              t[idx].astype(np.float64), n_out, width)
    assert float(loss) == pytest.approx(lr_, rel=2e-2)
    g = g.cpu().numpy()
    o, npad, total = M.layout(n_out, width)
    for k, (s, sh) in o.items():
        n = int(np.prod(sh))
        a, b = g[s:s + n], gr[s:s + n]
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b) + 1e-12, k


def test_adam_step_matches_the_oracle():
    d, p, net = _net(7, 64, 40, 32, 21)
    rng = np.random.default_rng(22)
    g = rng.normal(size=p.size).astype(np.float32)
    net.g.copy_(torch.from_numpy(g))
    m = np.zeros(p.size)
    v = np.zeros(p.size)
    pr = p.astype(np.float64)
    for step in range(1, 4):
        net.adam(1e-3)
        pr, m, v = M.adam(pr, m, v, g.astype(np.float64), step, 1e-3)
    np.testing.assert_allclose(net.p.cpu().numpy(), pr, rtol=0, atol=1e-6)
    q = net.q.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    np.testing.assert_array_equal(q.view(np.float32), M.bf16_round(net.p.cpu().numpy()))


def test_training_fits_a_teacher_network():
    n_in, width, n_out = 7, 128, 48
    d, p, net = _net(n_in, width, n_out, 128, 31)
    rng = np.random.default_rng(32)
    x = rng.uniform(-1, 1, size=(4096, n_in)).astype(np.float32)
    teacher = mlp.init_params(d, 99).astype(np.float64)
    t, _ = M.forward(teacher, x.astype(np.float64), n_out, width, rounding=False)
    t = (t / t.std()).astype(np.float32)
    X, T = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    losses = mlp.train(net, X, T, steps=1500, batch=128, lr=2e-3, seed=1)
    assert losses[-1] < 0.1 * losses[0]


def test_learned_warm_start_beats_the_cold_start():
    """The network trained (by these kernels) on the converged cold-start
    solutions of 32768 instances, against the plain cold start on 4096
    held-out instances: more of them converge within the iteration limit and
    the mean iteration count drops (the IPM from either starting point decides
    the result)."""
    from paper_2509_16370_b300 import inputs, ipm
    B = 4096
    model, opts = ipm.make_model(), ipm.make_ipm_opts()
    st = ipm.IpmState(B, model.N)
    ws = ipm.alloc_ipm_workspace(B, model, opts)
    feats, outs = [], []
    for s0 in range(0, 32768, B):
        x0, xg = inputs.workload5(B, s0)
        dx0, dxg = torch.from_numpy(x0).cuda(), torch.from_numpy(xg).cuda()
        ipm.rlqr_ipm_init(model, opts, dx0, st)
        ipm.rlqr_ipm_solve(model, opts, dx0, dxg, st, ws)
        ok = (st.status == ipm.CONVERGED).cpu().numpy()
        feats.append(mlp.features(x0[ok], xg[ok]))
        outs.append(mlp.targets(st.X.cpu().numpy()[ok], st.U.cpu().numpy()[ok]))
    F, T = np.concatenate(feats), np.concatenate(outs)
    norm = mlp.Normalizer(T)
    d = mlp.make_dims(mlp.N_IN, 256, T.shape[1], 256)
    net = mlp.WarmStartNet(d, mlp.init_params(d, 2025))
    mlp.train(net, torch.from_numpy(F).cuda(), torch.from_numpy(norm.encode(T)).cuda(),
              steps=4000, batch=256, lr=1e-3, lr_final=5e-5, seed=7)
    x0, xg = inputs.workload5(B, 2_000_000)
    dx0, dxg = torch.from_numpy(x0).cuda(), torch.from_numpy(xg).cuda()
    res = {}
    for kind in ("cold", "warm"):
        if kind == "cold":
            ipm.rlqr_ipm_init(model, opts, dx0, st)
        else:
            X0, U0 = mlp.propose(net, norm, x0, xg, model.N)
            ipm.rlqr_ipm_init(model, opts, dx0, st, U0=U0, X0=X0)
        ipm.rlqr_ipm_solve(model, opts, dx0, dxg, st, ws)
        conv = (st.status == ipm.CONVERGED).cpu().numpy()
        res[kind] = (conv.mean(), st.iters.double().mean().item())
    assert res["warm"][0] > 1.5 * res["cold"][0], res
    assert res["warm"][1] < res["cold"][1], res
