"""The warm-start network's CUDA kernels (BF16 tensor-core GEMMs with FP32
accumulation) against the FP64 oracle with BF16 rounding at the same points:
forward pass, loss and gradient, Adam step; and a short training run that
fits a teacher network.

Tolerances, element by element: the oracle accumulates in FP64 and the GPU
in FP32, and a value whose two sums straddle a BF16 rounding boundary rounds
to neighbouring BF16 values (relative spacing 2^-8) before the next layer.
Each output and gradient entry must agree within 2^-5 of its magnitude
scale -- the sum of the absolute values of the terms forming it
(oracle.mlp.abs_scales), i.e. a few BF16 ulps of each term -- plus an
absolute floor of 1e-6 of the block's largest scale; entries beyond that
(boundary-straddling outliers) are counted, reported, and limited to 0.5 %
of the block.  A planted mistake in the oracle (a dropped ReLU mask, a
transposed weight gradient) must fail the same comparison.  The Adam
arithmetic is exact up to FP32 rounding."""
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


REL_SCALE = 2.0 ** -5   # a few BF16 ulps (2^-8) of the terms' magnitude
OUTLIER_FRAC = 0.005


def elementwise(a, b, scale, name):
    """Element-wise agreement within REL_SCALE * scale + floor; returns the
    number of outliers after asserting it is at most OUTLIER_FRAC."""
    a, b, scale = (np.asarray(v, np.float64).ravel() for v in (a, b, scale))
    floor = 1e-6 * max(scale.max(), 1e-30)
    bad = np.abs(a - b) > REL_SCALE * scale + floor
    nbad = int(bad.sum())
    assert nbad <= max(1, OUTLIER_FRAC * a.size), \
        f"{name}: {nbad} of {a.size} entries outside the element-wise bound"
    return nbad


def _case(dims, seed=11):
    n_in, width, n_out, rows = dims
    d, p, net = _net(n_in, width, n_out, rows, seed)
    rng = np.random.default_rng(seed + 1)
    x = rng.normal(size=(rows * 2, n_in)).astype(np.float32)
    t = rng.normal(size=(rows * 2, n_out)).astype(np.float32)
    idx = rng.permutation(rows * 2)[:rows].astype(np.int32)
    return d, p, net, x, t, idx


def _gpu_grad(net, x, t, idx):
    loss, g = net.grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(),
                       torch.from_numpy(idx).cuda())
    return float(loss), g.cpu().numpy()


@pytest.mark.parametrize("dims", [(7, 64, 40, 32), (7, 256, 902, 64)])
def test_forward_and_gradient_match_the_oracle(dims):
    n_in, width, n_out, rows = dims
    d, p, net, x, t, idx = _case(dims)
    p64 = p.astype(np.float64)
    y = net.forward(torch.from_numpy(x[:rows]).cuda()).cpu().numpy()
    yr, _ = M.forward(p64, x[:rows].astype(np.float64), n_out, width)
    ys, _ = M.abs_scales(p64, x[:rows].astype(np.float64), np.zeros((rows, n_out)), n_out, width)
    report = {"y": elementwise(y, yr, ys, "forward")}
    loss, g = _gpu_grad(net, x, t, idx)
    xi, ti = x[idx].astype(np.float64), t[idx].astype(np.float64)
    lr_, gr = M.loss_and_grad(p64, xi, ti, n_out, width)
    _, gs = M.abs_scales(p64, xi, ti, n_out, width)
    assert loss == pytest.approx(lr_, rel=2e-2)
    o, npad, total = M.layout(n_out, width)
    for k, (s, sh) in o.items():
        n = int(np.prod(sh))
        report[k] = elementwise(g[s:s + n], gr[s:s + n], gs[s:s + n], k)
    print("outliers per block:", report)


def _mutated_grad(p, x, t, n_out, width, kind):
    """The oracle's gradient with one planted mistake (CPU only)."""
    r = M.bf16_round
    y, c = M.forward(p, x, n_out, width)
    rows = x.shape[0]
    npad = c["y"].shape[1]
    dy = np.zeros((rows, npad))
    dy[:, :n_out] = 2.0 * (y - t) / (rows * n_out)
    dy = r(dy)
    g = {"W3": dy.T @ c["h2"], "b3": dy.sum(axis=0)}
    mask2 = np.ones_like(c["h2"]) if kind == "relu" else (c["h2"] > 0)
    dz2 = r((dy @ c["P"]["W3"]) * mask2)
    g["W2"] = dz2.T @ c["h1"]
    if kind == "transpose":
        g["W2"] = g["W2"].T
    g["b2"] = dz2.sum(axis=0)
    dz1 = r((dz2 @ c["P"]["W2"]) * (c["h1"] > 0))
    g["W1"], g["b1"] = dz1.T @ c["a0"], dz1.sum(axis=0)
    return M.pack(g, n_out, width)


@pytest.mark.parametrize("kind", ["relu", "transpose"])
def test_elementwise_comparison_catches_a_planted_mistake(kind):
    """The element-wise criterion rejects the GPU gradient when the oracle
    carries a dropped ReLU mask or a transposed weight gradient."""
    dims = (7, 64, 40, 32)
    n_in, width, n_out, rows = dims
    d, p, net, x, t, idx = _case(dims)
    _, g = _gpu_grad(net, x, t, idx)
    p64 = p.astype(np.float64)
    xi, ti = x[idx].astype(np.float64), t[idx].astype(np.float64)
    bad = _mutated_grad(p64, xi, ti, n_out, width, kind)
    _, gs = M.abs_scales(p64, xi, ti, n_out, width)
    s, sh = M.layout(n_out, width)[0]["W2"]
    n = int(np.prod(sh))
    with pytest.raises(AssertionError):
        elementwise(g[s:s + n], bad[s:s + n], gs[s:s + n], "W2")


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


def test_graph_replayed_training_equals_eager_training():
    """mlp.train_graph (one captured step, batches and schedule read on the
    device) against mlp.train from the same start: bit-identical parameters,
    moments and losses after 320 steps over epoch boundaries with a decaying
    learning rate, and the step counters in agreement."""
    n_in, width, n_out = 7, 64, 40
    d, p, a = _net(n_in, width, n_out, 64, 41)
    _, _, b = _net(n_in, width, n_out, 64, 41)
    rng = np.random.default_rng(42)
    X = torch.from_numpy(rng.uniform(-1, 1, size=(1000, n_in)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(1000, n_out)).astype(np.float32)).cuda()
    la = mlp.train(a, X, T, steps=320, batch=64, lr=2e-3, seed=5, lr_final=1e-4)
    lb = mlp.train_graph(b, X, T, steps=320, batch=64, lr=2e-3, seed=5, lr_final=1e-4)
    torch.cuda.synchronize()
    assert la == lb
    for k in ("p", "q", "m", "v"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k
    assert a.step == b.step == 320


def test_checkpoint_resume_is_bit_exact(tmp_path):
    """Training that stops, saves its state (mlp.save_checkpoint), and goes
    on in a network restored from the file (mlp.load_checkpoint) ends with
    the parameters, Adam moments, BF16 copy and step counter bit-identical to
    the same training without the interruption."""
    n_in, width, n_out = 7, 64, 40
    d, p, a = _net(n_in, width, n_out, 64, 43)
    rng = np.random.default_rng(44)
    X = torch.from_numpy(rng.uniform(-1, 1, size=(700, n_in)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(700, n_out)).astype(np.float32)).cuda()
    mlp.train(a, X, T, steps=150, batch=64, lr=2e-3, seed=6)
    path = str(tmp_path / "net.npz")
    mlp.save_checkpoint(a, path)
    b = mlp.load_checkpoint(path)
    la = mlp.train(a, X, T, steps=120, batch=64, lr=1e-3, seed=7)
    lb = mlp.train(b, X, T, steps=120, batch=64, lr=1e-3, seed=7)
    torch.cuda.synchronize()
    assert la == lb
    for k in ("p", "q", "m", "v"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k
    assert a.step == b.step == 270


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
