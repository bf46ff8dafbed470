"""Pins of the oracle's regularized IPM (oracle/ipm.py) to things other than
itself (CPU only).

* the equations of motion against a symbolic Euler-Lagrange derivation of the
  cart with a double pendulum (sympy, from the kinetic and potential energy);
* the RK4 step: fourth-order convergence in the step size, and the energy of
  the frictionless model conserved to the method's error;
* second-order forward differentiation (Taylor2) against complex-step first
  derivatives and central differences of them;
* the Newton step through the dual-regularized LQR against the dense
  Newton-KKT system eq. ipm-4x4-newton-kkt solved by numpy, and the
  eigenvalue inertia of that system against the LQR certificate (Theorem
  inertia-al-descent's premise and the Section "Applying the regularized IPM
  to optimal control" theorem);
* the merit slope against a central difference of the merit, and against
  -[dx; ds]^T K_xs [dx; ds] (Lemma al-directional-derivative);
* a converged solve: every state is one RK4 step of the previous state and
  control, the Lagrangian gradient by finite differences vanishes, the bounds
  hold.
"""
import numpy as np
import pytest
import sympy as sp

import oracle.ipm as O
from paper_2509_16370_b300 import inputs


def _random_state(rng):
    return np.array([rng.uniform(-1, 1), rng.uniform(-np.pi, np.pi), rng.uniform(-np.pi, np.pi),
                     rng.normal(), 2 * rng.normal(), 2 * rng.normal()])


def test_equations_of_motion_match_euler_lagrange():
    md = O.Model()
    t = sp.symbols("t")
    p, a, b = (sp.Function(n)(t) for n in ("p", "a", "b"))
    u = sp.symbols("u")
    m0, m1, m2, l1, l2, g = (sp.Float(v) for v in (md.m0, md.m1, md.m2, md.l1, md.l2, md.grav))
    x1, y1 = p + l1 * sp.sin(a), l1 * sp.cos(a)
    x2, y2 = x1 + l2 * sp.sin(b), y1 + l2 * sp.cos(b)
    d = lambda e: sp.diff(e, t)  # noqa: E731
    T = (m0 * d(p) ** 2 + m1 * (d(x1) ** 2 + d(y1) ** 2) + m2 * (d(x2) ** 2 + d(y2) ** 2)) / 2
    V = m1 * g * y1 + m2 * g * y2
    L = T - V
    q = [p, a, b]
    forces = [u, 0, 0]
    eqs = [d(sp.diff(L, d(qi))) - sp.diff(L, qi) - f for qi, f in zip(q, forces)]
    acc = [sp.diff(qi, t, 2) for qi in q]
    Mm = sp.Matrix([[sp.diff(e, ai) for ai in acc] for e in eqs])
    rest = sp.Matrix([e.subs({ai: 0 for ai in acc}) for e in eqs])
    syms = sp.symbols("P A Bb dP dA dB")
    sub = {sp.diff(qi, t): s for qi, s in zip(q, syms[3:])}
    sub2 = {qi: s for qi, s in zip(q, syms[:3])}
    fM = sp.lambdify([*syms, u], Mm.subs(sub).subs(sub2), "numpy")
    fr = sp.lambdify([*syms, u], rest.subs(sub).subs(sub2), "numpy")
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = _random_state(rng)
        uu = rng.uniform(-20, 20)
        qdd = np.linalg.solve(np.array(fM(*x, uu), float), -np.array(fr(*x, uu), float).ravel())
        f = O.rhs(md, list(x), uu)
        np.testing.assert_allclose(f[:3], x[3:], rtol=0, atol=0)
        np.testing.assert_allclose(f[3:], qdd, rtol=1e-12, atol=1e-12)


def _integrate(md, x, u, T, dt):
    m = O.Model(dt=dt)
    X = np.asarray(x, float)[None, :]
    for _ in range(int(round(T / dt))):
        X = O.step_map(m, X, np.array([u]))
    return X[0]


def test_rk4_is_fourth_order_and_conserves_energy():
    md = O.Model()
    x = np.array([0.0, 2.5, -1.0, 0.0, 0.5, -0.3])
    ref = _integrate(md, x, 0.0, 0.64, 0.02 / 128)
    e1 = np.abs(_integrate(md, x, 0.0, 0.64, 0.005) - ref).max()
    e2 = np.abs(_integrate(md, x, 0.0, 0.64, 0.0025) - ref).max()
    assert 13.0 < e1 / e2 < 19.0          # 2^4 = 16 for a fourth-order method
    # energy drift of the frictionless model under u = 0 over 128 steps:
    # small at dt = 0.02 and shrinking like the method's error with the step
    drift = []
    for dt in (0.02, 0.005, 0.0025):
        X = O.rollout(O.Model(dt=dt, N=int(round(2.56 / dt))), x, np.zeros(int(round(2.56 / dt))))
        E = np.array([O.energy(md, xi) for xi in X])
        drift.append(np.abs(E - E[0]).max() / abs(E[0]))
    assert drift[0] <= 2e-3
    assert drift[1] / drift[2] > 10.0


def test_taylor2_derivatives_match_complex_step_and_differences():
    md = O.Model()
    rng = np.random.default_rng(1)
    S = 5
    w = np.stack([np.concatenate([_random_state(rng), [rng.uniform(-5, 5)]]) for _ in range(S)])
    v = O.Taylor2.variables(w)
    phi = O.rk4(md, v[:6], v[6])
    h = 1e-30
    for k in range(7):
        wc = w.astype(complex)
        wc[:, k] += 1j * h
        out = O.rk4(md, [wc[:, j] for j in range(6)], wc[:, 6])
        for l in range(6):
            np.testing.assert_allclose(phi[l].g[:, k], out[l].imag / h, rtol=1e-12, atol=1e-13)

    def grad(wv):
        res = np.zeros((S, 6, 7))
        for k in range(7):
            wc = wv.astype(complex)
            wc[:, k] += 1j * h
            out = O.rk4(md, [wc[:, j] for j in range(6)], wc[:, 6])
            res[:, :, k] = np.stack([o.imag / h for o in out], axis=1)
        return res
    e = 1e-5
    for k in range(7):
        dw = np.zeros_like(w)
        dw[:, k] = e
        fd = (grad(w + dw) - grad(w - dw)) / (2 * e)
        for l in range(6):
            np.testing.assert_allclose(phi[l].h[:, :, k], fd[:, l, :], rtol=1e-6, atol=1e-7)


def _perturbed_state(md, op, seed, b=2):
    rng = np.random.default_rng(seed)
    x0, xg = inputs.workload5_instance(b)
    st = O.initial_state(md, op, x0, xg, U=3 * rng.standard_normal(md.N))
    st.X += 0.05 * rng.standard_normal(st.X.shape)
    st.Y = rng.standard_normal(st.Y.shape)
    m = O.inequalities(md, st.X, st.U)[1]
    st.Z = np.where(m, rng.uniform(0.05, 1.0, st.Z.shape), 0.0)
    st.S = np.where(m, rng.uniform(0.1, 2.0, st.S.shape), 1.0)
    st.mu = 0.05
    return st


@pytest.mark.parametrize("exact", [True, False])
def test_lqr_route_solves_the_dense_newton_kkt_system(exact):
    md, op = O.Model(N=10), O.Options(exact_hessian=exact)
    st = _perturbed_state(md, op, 3)
    lin = O.linearize(md, op, st)
    for rho in (0.0, 0.7):
        res, _, dX, dU, dS, dY, dZ, _ = O.newton_lqr(md, op, st, lin, rho)
        assert res.status < 2
        d = O.newton_dense(md, op, st, lin, rho)
        for a, ref in ((dX, d["dX"]), (dU, d["dU"]), (dS, d["dS"]), (dY, d["dY"]), (dZ, d["dZ"])):
            np.testing.assert_allclose(a, ref, rtol=0, atol=1e-9 * max(1, np.abs(ref).max()))
        # the dense system itself: residual of numpy's solution
        sol = np.concatenate([_flat(md, d["dX"], d["dU"]), d["dS"][lin.mask],
                              d["dY"].ravel(), d["dZ"][lin.mask]])
        assert np.abs(d["K"] @ sol - d["rhs"]).max() <= 1e-10 * np.abs(d["rhs"]).max()


def _flat(md, dX, dU):
    out = []
    for i in range(md.N):
        out += list(dX[i]) + [dU[i]]
    return np.array(out + list(dX[md.N]))


def _inertia(K):
    ev = np.linalg.eigvalsh(K)
    tol = 1e-9 * np.abs(ev).max()
    return int((ev > tol).sum()), int((ev < -tol).sum()), int((np.abs(ev) <= tol).sum())


def test_certificate_matches_the_eigenvalue_inertia_of_the_newton_system():
    """All LQR pivot flags PD <=> In(K_4) = (n_x + n_g, n_c + n_g, 0), on
    states whose exact Hessian has both outcomes."""
    md, op = O.Model(N=12), O.Options()
    seen = set()
    for seed in range(20):
        st = _perturbed_state(md, op, 100 + seed)
        st.Y *= 120.0                                # large duals: both outcomes occur
        lin = O.linearize(md, op, st)
        res, *_ = O.newton_lqr(md, op, st, lin, 0.0)
        d = O.newton_dense(md, op, st, lin, 0.0)
        nx = md.N * 7 + 6
        ng = int(lin.mask.sum())
        nc = (md.N + 1) * 6
        ok = bool(np.all(res.flags == 3))
        assert (_inertia(d["K"]) == (nx + ng, nc + ng, 0)) == ok
        seen.add(ok)
    assert seen == {True, False}


def test_merit_slope_matches_differences_and_the_kxs_form():
    md, op = O.Model(N=10), O.Options()
    st = _perturbed_state(md, op, 7)
    lin = O.linearize(md, op, st)
    rho = 50.0                                      # ensures the correct inertia
    res, _, dX, dU, dS, dY, dZ, Gdx = O.newton_lqr(md, op, st, lin, rho)
    assert np.all(res.flags == 3)
    slope = O.merit_slope(md, op, st, lin, dX, dU, dS, Gdx)
    m = lin.mask
    f = lambda a: O.merit(md, op, st, st.X + a * dX, st.U + a * dU,  # noqa: E731
                          np.where(m, st.S + a * dS, 1.0), st.mu)
    e = 1e-6
    assert slope == pytest.approx((f(e) - f(-e)) / (2 * e), rel=1e-6)
    # Lemma al-directional-derivative: slope = -[dx; ds]^T K_xs [dx; ds]
    d = O.newton_dense(md, op, st, lin, rho)
    ng = int(m.sum())
    dxv, dsv = _flat(md, dX, dU), dS[m]
    W_inv = np.diag(st.Z[m] / st.S[m])
    Cx = d["C"] @ dxv
    Gx = d["G"] @ dxv
    quad = dxv @ d["P"] @ dxv + dsv @ W_inv @ dsv + op.eta * (Cx @ Cx) + \
        op.eta * ((Gx + dsv) @ (Gx + dsv))
    assert slope == pytest.approx(-quad, rel=1e-8)
    assert slope < 0 and ng > 0


def test_converged_solve_is_a_kkt_point():
    """A swing-up instance the oracle solves to the tolerance (instance 5 of
    the workload): the final controls roll out to the final states, the
    Lagrangian's gradient (central differences) vanishes, the bounds hold and
    the complementarity is below the tolerance."""
    md, op = O.Model(), O.Options()
    x0, xg = inputs.workload5_instance(5)
    st = O.solve(md, op, x0, xg)
    assert st.status == 1
    # one RK4 step from every final state with its control lands on the next
    # state (a full rollout would amplify the 1e-6 defects: the upright
    # pendulum is unstable)
    one = O.Model(N=1)
    for i in range(md.N):
        nxt = O.rollout(one, st.X[i], st.U[i:i + 1])[1]
        assert np.abs(nxt - st.X[i + 1]).max() <= op.tol
    assert np.abs(st.X[0] - x0).max() <= op.tol
    g, m = O.inequalities(md, st.X, st.U)
    assert np.all(g[m] <= 1e-6)
    assert np.all((st.S * st.Z)[m] <= op.tol)

    def lagr(X, U):
        gg, mm = O.inequalities(md, X, U)
        c = O.defects(md, x0, X, U)
        return O.cost(md, X, U, xg) + np.sum(st.Y * c) + np.sum((st.Z * (gg + st.S))[mm])
    h = 1e-6
    worst = 0.0
    for i in range(0, md.N + 1, 16):
        for j in range(6):
            Xp, Xm = st.X.copy(), st.X.copy()
            Xp[i, j] += h
            Xm[i, j] -= h
            worst = max(worst, abs(lagr(Xp, st.U) - lagr(Xm, st.U)) / (2 * h))
    assert worst <= 1e-5
