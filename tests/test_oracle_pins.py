"""Pins of the FP64 oracle to things other than itself.

Each test ties an oracle function to the paper's printed examples, to exact
rational arithmetic on the Lagrangian's definition, to closed forms, to a
library routine (numpy / scipy), or to an invariant stated by a theorem.
Chosen so that a dropped term, a wrong sign or index, or a transposed operand
anywhere in the oracle fails at least one of them.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg
import sympy as sp

import oracle
from paper_2509_16370_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        d = json.load(f)
    arr = {k: np.array(d[k], dtype=np.float64) for k in ("Q", "M", "R", "q", "r", "A", "B", "c")}
    return d, inputs.Problem(d["N"], d["n"], d["m"], delta=float(d["delta"]), **arr)


# ------------------------------------------------------- worked examples

def test_worked_example_1_matrix_and_solution():
    """The two-stage example without dual regularization: the assembled KKT
    matrix and right-hand side equal the printed ones, and every solver
    returns the printed solution (0, 0, -1, 0, -3)."""
    d, p = _load("worked_example_1.json")
    K, b = oracle.kkt_dense(p)
    np.testing.assert_array_equal(K, np.array(d["printed_K"], float))
    np.testing.assert_array_equal(-b, np.array(d["printed_rhs"], float))
    want = np.array(d["printed_solution"]["value"], float)
    r = oracle.riccati(p)
    assert r.status == oracle.OK
    z = oracle.join_solution(p, r.x, r.u, r.y)
    np.testing.assert_allclose(z, want, atol=1e-15)
    x, u, y, inertia = oracle.dense_solve(p)
    np.testing.assert_allclose(oracle.join_solution(p, x, u, y), want, atol=1e-15)
    st, x, u, y = oracle.band_solve(p)
    assert st == 0
    np.testing.assert_allclose(oracle.join_solution(p, x, u, y), want, atol=1e-15)
    assert oracle.residual(p, r.x, r.u, r.y).rmax == 0.0


def test_worked_example_1_merit_slope():
    """The example's directional derivative equals 2 - eta for the printed
    step (reading: the display's 1/2 on the primal quadratic is a typo, since
    grad f^T dx = -1, y^T C dx = 3 and eta c^T C dx = -eta give 2 - eta)."""
    d, p = _load("worked_example_1.json")
    dz = np.array(d["printed_solution"]["value"], float)
    dx, dy = dz[:3], dz[3:]
    grad_f = np.array([0.0, 0.0, 1.0])  # f = (x0^2 + u0^2 + x1^2)/2 at (0, 0, 1)
    C = np.array([[-1.0, 0, 0], [1.0, 1.0, -1.0]])
    y = np.array([0.0, 3.0])
    c_val = np.array([0.0, -1.0])  # c(x) = (s0 - x0, x0 + u0 - x1) at (0, 0, 1)
    assert dy.shape == (2,)
    for eta in (0.5, 2.0, 7.0):
        # derivative of f + y^T c + (eta/2)||c||^2 along the primal step only
        # (Lemma al-directional-derivative-lemma): (grad f + C^T y + eta C^T c)^T dx
        slope = grad_f @ dx + y @ (C @ dx) + eta * c_val @ (C @ dx)
        assert slope == pytest.approx(2.0 - eta, abs=1e-14)


def test_worked_example_2_inertia_and_pivots():
    """The scalar example with an indefinite stage Hessian: P, C and
    P + C^T C match the printed matrices, the leading minors are 2, 6, 4, the
    inertia is (3, 2, 0), and the recursion's pivots are PD with
    S_1 = 2, G_0 = 1, S_0 = 2 (product 4 = det(P + C^T C))."""
    d, p = _load("worked_example_2.json")
    K, b = oracle.kkt_dense(p)
    nxp, nyd = oracle.kkt_dims(p.N, p.n, p.m)
    Pm, Cm = K[:nxp, :nxp], K[nxp:, :nxp]
    np.testing.assert_array_equal(Pm, np.array(d["printed_P"], float))
    np.testing.assert_array_equal(Cm, np.array(d["printed_C"], float))
    PCC = Pm + Cm.T @ Cm / p.delta
    np.testing.assert_array_equal(PCC, np.array(d["printed_P_plus_CtC"], float))
    minors = [np.linalg.det(PCC[:k, :k]) for k in (1, 2, 3)]
    np.testing.assert_allclose(minors, d["printed_leading_minors"], rtol=1e-14)
    assert oracle.bk_inertia(oracle.bk_factor(K)) == tuple(d["printed_inertia"])
    assert oracle.jacobi_inertia(K)[0] == tuple(d["printed_inertia"])
    r = oracle.riccati(p, internals=True)
    assert r.status == oracle.OK and list(r.flags) == [3, 3]
    # S_i = P_i + Delta^{-1}; with delta = 1 the inverse-free S-hat equals S.
    np.testing.assert_allclose(r.S[:, 0, 0], [2.0, 2.0], rtol=1e-15)
    np.testing.assert_allclose(r.G[:, 0, 0], [1.0], rtol=1e-15)
    assert r.S[0, 0, 0] * r.G[0, 0, 0] * r.S[1, 0, 0] == pytest.approx(4.0)
    x, u, y, _ = oracle.dense_solve(p)
    assert oracle.forward_error((x, u, y), r.x, r.u, r.y) < 1e-15


# ------------------------------------------- exact rational pins (sympy)

def _rational_problem(seed, N, n, m, delta):
    rng = np.random.default_rng(seed)
    ri = lambda *s: rng.integers(-3, 4, size=s).astype(float)  # noqa: E731
    Q = ri(N + 1, n, n)
    Q = Q + np.swapaxes(Q, 1, 2) + 6 * np.eye(n)
    R = ri(N, m, m)
    R = R + np.swapaxes(R, 1, 2) + 8 * np.eye(m)
    return inputs.Problem(N, n, m, Q=Q, M=ri(N, n, m), R=R, q=ri(N + 1, n), r=ri(N, m),
                          A=ri(N, n, n), B=ri(N, n, m), c=ri(N + 1, n), delta=float(delta))


def _lagrangian_solution(p):
    """Exact solution from eq. min-max-with-ys: build the saddle function R as
    a polynomial in the unknowns, set its gradient to zero and solve with
    rational arithmetic.  Returns (Hessian, gradient at 0, solution) in the
    unknown order x_0, u_0, ..., x_N, y_0, ..., y_N."""
    N, n, m = p.N, p.n, p.m
    F = lambda v: sp.Rational(Fraction(float(v)).limit_denominator(1 << 20))  # noqa: E731
    xs = [sp.Matrix(sp.symbols(f"x{i}_0:{n}")) for i in range(N + 1)]
    us = [sp.Matrix(sp.symbols(f"u{i}_0:{m}")) for i in range(N)]
    ys = [sp.Matrix(sp.symbols(f"y{i}_0:{n}")) for i in range(N + 1)]
    mat = lambda a: sp.Matrix([[F(v) for v in row] for row in np.atleast_2d(a)])  # noqa: E731
    vec = lambda a: sp.Matrix([F(v) for v in np.ravel(a)])  # noqa: E731
    delta = F(p.delta)
    Rf = 0
    for i in range(N):
        Qi, Mi, Ri = mat(p.Q[i]), mat(p.M[i]), mat(p.R[i])
        Rf += (sp.Rational(1, 2) * (xs[i].T * Qi * xs[i])[0] + (xs[i].T * Mi * us[i])[0]
               + sp.Rational(1, 2) * (us[i].T * Ri * us[i])[0] + (vec(p.q[i]).T * xs[i])[0]
               + (vec(p.r[i]).T * us[i])[0])
        dyn = mat(p.A[i]) * xs[i] + mat(p.B[i]) * us[i] + vec(p.c[i + 1]) - xs[i + 1]
        Rf += (ys[i + 1].T * dyn)[0]
    Rf += sp.Rational(1, 2) * (xs[N].T * mat(p.Q[N]) * xs[N])[0] + (vec(p.q[N]).T * xs[N])[0]
    for i in range(N + 1):
        Rf -= sp.Rational(1, 2) * delta * (ys[i].T * ys[i])[0]
    Rf += (ys[0].T * (vec(p.c[0]) - xs[0]))[0]
    unknowns = []
    for i in range(N + 1):
        unknowns += list(xs[i])
        if i < N:
            unknowns += list(us[i])
    for i in range(N + 1):
        unknowns += list(ys[i])
    grad = sp.Matrix([sp.diff(Rf, v) for v in unknowns])
    H = grad.jacobian(unknowns)
    g0 = grad.subs({v: 0 for v in unknowns})
    sol = H.LUsolve(-g0)
    return H, g0, sol


@pytest.mark.parametrize("seed,N,n,m,delta", [
    (1, 1, 1, 1, 0.0), (2, 2, 2, 1, 0.5), (3, 3, 2, 2, 1.0), (4, 2, 1, 2, 0.25),
    (5, 3, 2, 1, 0.0)])
def test_exact_rational_lagrangian(seed, N, n, m, delta):
    """The oracle's KKT assembly equals the exact Hessian of the saddle
    function of eq. min-max-with-ys, its right-hand side equals the exact
    gradient at zero, and the recursion, dense and banded solvers all return
    the exact rational solution (to FP64 rounding)."""
    p = _rational_problem(seed, N, n, m, delta)
    H, g0, sol = _lagrangian_solution(p)
    K, b = oracle.kkt_dense(p)
    np.testing.assert_array_equal(K, np.array(H.tolist(), dtype=float))
    np.testing.assert_array_equal(b, np.array(g0.tolist(), dtype=float).ravel())
    exact = np.array([float(v) for v in sol])
    scale = np.abs(exact).max()
    r = oracle.riccati(p)
    assert r.status in (oracle.OK, oracle.NOT_PD)
    assert np.abs(oracle.join_solution(p, r.x, r.u, r.y) - exact).max() <= 1e-12 * scale
    x, u, y, _ = oracle.dense_solve(p)
    assert np.abs(oracle.join_solution(p, x, u, y) - exact).max() <= 1e-12 * scale
    st, x, u, y = oracle.band_solve(p)
    assert np.abs(oracle.join_solution(p, x, u, y) - exact).max() <= 1e-12 * scale


# ------------------------------------------------------- closed forms

def test_scalar_steady_state_closed_form():
    """n = m = 1, M = 0, time-invariant data: P_0 of a long horizon equals
    W/(1 - delta W), W the positive root of
    (b^2 + delta(q b^2 + a^2 r)) W^2 + (r - q b^2 - a^2 r + delta q r) W - q r = 0,
    which is the fixed point of W = P/(1 + delta P), P = q + a^2 r W / (r + b^2 W)
    (our derivation from eq. value-fn-formulas); at delta = 0 it is the
    textbook scalar DARE."""
    N = 4000
    for a, bb, qq, rr, delta in [(0.9, 0.7, 2.0, 0.5, 0.3), (1.3, 1.1, 1.0, 2.0, 1e-3),
                                 (0.5, 2.0, 3.0, 0.1, 0.0), (1.05, 0.4, 0.7, 1.5, 2.0)]:
        p = inputs.Problem(N, 1, 1, Q=np.full((N + 1, 1, 1), qq), M=np.zeros((N, 1, 1)),
                           R=np.full((N, 1, 1), rr), q=np.zeros((N + 1, 1)), r=np.zeros((N, 1)),
                           A=np.full((N, 1, 1), a), B=np.full((N, 1, 1), bb),
                           c=np.zeros((N + 1, 1)), delta=delta)
        res = oracle.riccati(p, internals=True)
        c2 = bb * bb + delta * (qq * bb * bb + a * a * rr)
        c1 = rr - qq * bb * bb - a * a * rr + delta * qq * rr
        c0 = -qq * rr
        W = (-c1 + np.sqrt(c1 * c1 - 4 * c2 * c0)) / (2 * c2)
        P_inf = W / (1 - delta * W)
        assert res.P[0, 0, 0] == pytest.approx(P_inf, rel=1e-13)


def test_delta_zero_matches_scipy_dare_with_cross_term():
    """delta = 0 reduces the recursion to the standard Riccati recursion
    (W = P); with time-invariant data P_0 of a long horizon equals scipy's
    DARE solution, cross term M included."""
    rng = inputs.rng_for(97, 0)
    n, m, N = 4, 2, 3000
    A = inputs.spectral_rescaled(rng, 1, n, 1.1)[0]
    B = rng.standard_normal((n, m))
    Q = inputs.llt_plus(rng, 1, n, 0.5)[0]
    R = inputs.llt_plus(rng, 1, m, 0.5)[0]
    M = 0.1 * rng.standard_normal((n, m))
    p = inputs.Problem(N, n, m, Q=np.broadcast_to(Q, (N + 1, n, n)).copy(),
                       M=np.broadcast_to(M, (N, n, m)).copy(),
                       R=np.broadcast_to(R, (N, m, m)).copy(), q=np.zeros((N + 1, n)),
                       r=np.zeros((N, m)), A=np.broadcast_to(A, (N, n, n)).copy(),
                       B=np.broadcast_to(B, (N, n, m)).copy(), c=np.zeros((N + 1, n)),
                       delta=0.0)
    res = oracle.riccati(p, internals=True)
    X = scipy.linalg.solve_discrete_are(A, B, Q, R, s=M)
    np.testing.assert_allclose(res.P[0], X, rtol=1e-10, atol=1e-10)
    # delta = 0: x_0 = c_0 exactly (eq. recover-x0 with Delta_0 = 0)
    assert np.array_equal(res.x[0], p.c[0])


def test_delta_to_zero_limit():
    """The solution is a rational function of delta that is regular at 0, so
    the error to the delta = 0 (standard LQR) solution shrinks linearly."""
    base = inputs.random_instance(11, 20, 3, 2, 0.0)
    ref = oracle.riccati(base)
    errs = []
    for delta in (1e-3, 1e-4, 1e-5, 1e-6):
        p = inputs.random_instance(11, 20, 3, 2, delta)
        r = oracle.riccati(p)
        errs.append(oracle.forward_error((ref.x, ref.u, ref.y), r.x, r.u, r.y))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    for rt in ratios:
        assert 8.0 < rt < 12.5
    assert errs[-1] < 1e-4


# ------------------------------------------------- library cross-checks

@pytest.mark.parametrize("seed,N,n,m,delta,withM", [
    (0, 5, 3, 2, 1e-2, True), (1, 9, 4, 1, 1e-6, True), (2, 3, 2, 3, 0.0, True),
    (3, 12, 5, 2, 1.0, False), (4, 6, 1, 1, 3.0, True)])
def test_recursion_matches_numpy_solve(seed, N, n, m, delta, withM):
    """The recursion's (x, u, y) equals numpy.linalg.solve of the assembled
    system; nonsymmetric A, M != 0 and delta = 0 included."""
    p = inputs.random_instance(seed, N, n, m, delta, with_M=withM)
    K, b = oracle.kkt_dense(p)
    zn = np.linalg.solve(K, -b)
    r = oracle.riccati(p)
    assert r.status in (oracle.OK, oracle.NOT_PD)
    assert oracle.forward_error(oracle.split_solution(p, zn), r.x, r.u, r.y) < 1e-11
    x, u, y, _ = oracle.dense_solve(p)
    assert oracle.forward_error(oracle.split_solution(p, zn), x, u, y) < 1e-11
    st, x, u, y = oracle.band_solve(p)
    assert st == 0
    assert oracle.forward_error(oracle.split_solution(p, zn), x, u, y) < 1e-11


def test_bunch_kaufman_on_indefinite_matrices():
    """Bunch-Kaufman solve and inertia against numpy on symmetric indefinite
    matrices, including ones with a zero diagonal that force 2x2 pivots."""
    rng = np.random.default_rng(5)
    for dim in (1, 2, 5, 17, 40):
        for kind in ("dense", "zero_diag", "saddle"):
            X = rng.standard_normal((dim, dim))
            S = X + X.T
            if kind == "zero_diag":
                np.fill_diagonal(S, 0.0)
            if kind == "saddle" and dim >= 2:
                h = dim // 2
                S[:h, :h] = 0.0
            if abs(np.linalg.det(S)) < 1e-8:
                continue
            fac = oracle.bk_factor(S)
            rhs = rng.standard_normal(dim)
            np.testing.assert_allclose(oracle.bk_solve(fac, rhs), np.linalg.solve(S, rhs),
                                       rtol=1e-9, atol=1e-9)
            ev = np.linalg.eigvalsh(S)
            assert oracle.bk_inertia(fac) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
            if kind == "zero_diag" and dim >= 2:
                assert (fac[2] == 2).any()


def test_jacobi_inertia_matches_eigvalsh():
    rng = np.random.default_rng(6)
    for dim in (3, 10, 33):
        X = rng.standard_normal((dim, dim))
        S = X + X.T
        (pos, neg, zer), eig = oracle.jacobi_inertia(S)
        ev = np.linalg.eigvalsh(S)
        np.testing.assert_allclose(np.sort(eig), ev, atol=1e-10)
        assert (pos, neg, zer) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)


def test_residual_formula_equals_assembled_product():
    """The stagewise residual of Section "Residual Computation" equals K z + b
    computed from the assembled matrix for an arbitrary z, and its norms equal
    the assembled matrix's infinity norms."""
    p = inputs.random_instance(21, 6, 3, 2, 0.37)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((p.N + 1, p.n))
    u = rng.standard_normal((p.N, p.m))
    y = rng.standard_normal((p.N + 1, p.n))
    res = oracle.residual(p, x, u, y)
    K, b = oracle.kkt_dense(p)
    full = K @ oracle.join_solution(p, x, u, y) + b
    nxp, _ = oracle.kkt_dims(p.N, p.n, p.m)
    fx, fu, fy = oracle.split_solution(p, full)
    np.testing.assert_allclose(res.res_q, fx, atol=1e-13)
    np.testing.assert_allclose(res.res_r, fu, atol=1e-13)
    np.testing.assert_allclose(res.res_c, fy, atol=1e-13)
    assert res.rmax == pytest.approx(np.abs(full).max(), rel=1e-14)
    assert res.kmax == pytest.approx(np.abs(K).sum(axis=1).max(), rel=1e-14)
    assert res.bmax == pytest.approx(np.abs(b).max(), rel=1e-14)
    z = oracle.join_solution(p, x, u, y)
    assert res.zmax == pytest.approx(np.abs(z).max(), rel=1e-14)
    assert res.rel == pytest.approx(res.rmax / (res.kmax * res.zmax + res.bmax), rel=1e-14)


# --------------------------------------------------------- invariants

def _cases():
    out = [inputs.random_instance(s, 8, 3, 2, d, with_M=True) for s, d in
           ((31, 1e-2), (32, 0.5), (33, 2.0), (34, 1e-4))]
    # non-convex: a Q with negative eigenvalues and an indefinite R
    p = inputs.random_instance(35, 8, 3, 2, 0.3, with_M=True)
    p.Q[3] -= 4.0 * np.eye(3)
    p.R[5] -= 3.0 * np.eye(2)
    out.append(p)
    return out


@pytest.mark.parametrize("idx", range(5))
def test_inertia_identity(idx):
    """Theorem riccati-inertia-certification-theorem and its proof: with
    Delta = delta I > 0 the number of negative eigenvalues of K_LQR is
    (N+1) n + (negative pivots of all I + delta P_i and G_i).  BK, Jacobi and
    numpy all agree, and 'all flags PD' holds iff the inertia is
    (N(n+m)+n, (N+1)n, 0)."""
    p = _cases()[idx]
    r = oracle.riccati(p, internals=True)
    K, _ = oracle.kkt_dense(p)
    ev = np.linalg.eigvalsh(K)
    want_neg = (p.N + 1) * p.n + int(r.neg_S.sum()) + int(r.neg_G.sum())
    dim = K.shape[0]
    assert int((ev < 0).sum()) == want_neg
    assert oracle.bk_inertia(oracle.bk_factor(K)) == (dim - want_neg, want_neg, 0)
    assert oracle.jacobi_inertia(K)[0] == (dim - want_neg, want_neg, 0)
    nxp, nyd = oracle.kkt_dims(p.N, p.n, p.m)
    all_pd = bool((r.flags == 3).all())
    assert all_pd == (want_neg == nyd)
    assert (r.status == oracle.OK) == all_pd
    # flag bits are exactly the negative-count tests
    assert list(r.flags[:-1] & 1) == [int(v == 0) for v in r.neg_S[:-1]]
    assert list((r.flags[:-1] >> 1) & 1) == [int(v == 0) for v in r.neg_G]
    # pivot eigenvalues (numpy) agree with the LDL^T negative counts
    for i in range(p.N + 1):
        assert int((np.linalg.eigvalsh(r.S[i]) < 0).sum()) == r.neg_S[i]
    for i in range(p.N):
        assert int((np.linalg.eigvalsh(r.G[i]) < 0).sum()) == r.neg_G[i]


def test_p_recurrence_and_psd():
    """Corollary p-recurrence: p_k = q_k + K_k^T r_k + (A_k + B_k K_k)^T
    (p_{k+1} + W_{k+1}(c_{k+1} - delta p_{k+1})), with W = P (I + delta P)^{-1}
    formed here by numpy; and P_k is PSD on convex data (the Schur-complement
    argument after eq. value-fn-formulas)."""
    p = inputs.random_instance(41, 15, 4, 2, 0.05, with_M=False)
    r = oracle.riccati(p, internals=True)
    I = np.eye(p.n)
    for k in range(p.N):
        Pn = r.P[k + 1]
        W = np.linalg.solve((I + p.delta * Pn).T, Pn.T).T
        g = r.p[k + 1] + W @ (p.c[k + 1] - p.delta * r.p[k + 1])
        want = p.q[k] + r.K[k].T @ p.r[k] + (p.A[k] + p.B[k] @ r.K[k]).T @ g
        np.testing.assert_allclose(r.p[k], want, rtol=1e-12, atol=1e-12)
        assert np.linalg.eigvalsh(r.P[k]).min() > -1e-12 * np.abs(r.P[k]).max()
    # the costate identity y_k = Delta^{-1}(A x + B u + c - x_{k+1}) of eq. recover-y
    for k in range(p.N):
        lhs = r.y[k + 1] * p.delta
        rhs = p.A[k] @ r.x[k] + p.B[k] @ r.u[k] + p.c[k + 1] - r.x[k + 1]
        np.testing.assert_allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("mutation", ["transpose_A", "drop_M", "flip_c", "drop_delta",
                                      "transpose_B_rows"])
def test_pins_detect_planted_mistakes(mutation):
    """Sensitivity of the pins: feeding the oracle's recursion a plausibly
    wrong reading of the data (a transposed A, a dropped M, a sign flip on c, a
    dropped delta) moves its answer far from numpy's solve of the true system,
    so the cross-checks above would catch such a mistake."""
    p = inputs.random_instance(51, 6, 3, 2, 0.2, with_M=True)
    K, b = oracle.kkt_dense(p)
    truth = oracle.split_solution(p, np.linalg.solve(K, -b))
    bad = inputs.Problem(p.N, p.n, p.m, delta=p.delta, **{k: v.copy() for k, v in
                                                          p.arrays().items()})
    if mutation == "transpose_A":
        bad.A = np.ascontiguousarray(np.swapaxes(bad.A, 1, 2))
    elif mutation == "drop_M":
        bad.M[:] = 0.0
    elif mutation == "flip_c":
        bad.c = -bad.c
    elif mutation == "drop_delta":
        bad.delta = 0.0
    elif mutation == "transpose_B_rows":
        bad.B = bad.B[:, ::-1, :].copy()
    r = oracle.riccati(bad)
    assert oracle.forward_error(truth, r.x, r.u, r.y) > 1e-3
    assert oracle.residual(p, r.x, r.u, r.y).rel > 1e-6


# ------------------------------------------- cross-stage variables

def _cross_terms(seed, prob, p_theta):
    rng = np.random.default_rng(seed)
    N, n, m = prob.N, prob.n, prob.m
    ri = lambda *s: rng.integers(-2, 3, size=s).astype(float)  # noqa: E731
    Hs = ri(p_theta, p_theta)
    H = Hs + Hs.T + 5 * np.eye(p_theta)
    return ri(p_theta, N + 1, n), ri(p_theta, N, m), ri(p_theta, N + 1, n), H, ri(p_theta)


@pytest.mark.parametrize("seed,N,n,m,delta,p_theta", [(21, 2, 2, 1, 0.5, 1), (22, 2, 1, 1, 1.0, 2),
                                                       (23, 1, 2, 1, 0.25, 2)])
def test_cross_stage_exact_rational(seed, N, n, m, delta, p_theta):
    """Section "Cross-Stage Variables": the saddle function of eq.
    min-max-with-ys extended by theta^T J^T w + theta^T H theta / 2 +
    r_theta^T theta (J's (q, r, c) parts paired with (x, u, y)) has the
    Hessian [[K, J], [J^T, H]] and the gradient [b; r_theta] at zero; its
    exact rational stationary point equals the oracle's bordered solve."""
    prob = _rational_problem(seed, N, n, m, delta)
    Jq, Jr, Jc, H, rt = _cross_terms(seed, prob, p_theta)
    F = lambda v: sp.Rational(Fraction(float(v)).limit_denominator(1 << 20))  # noqa: E731
    Hw, g0, _ = _lagrangian_solution(prob)
    # unknown order of _lagrangian_solution: x_0, u_0, ..., x_N, y_0, ..., y_N
    J = sp.Matrix([[F(v) for v in oracle.join_solution(prob, Jq[j], Jr[j], Jc[j])]
                   for j in range(p_theta)]).T
    Hb = Hw.row_join(J).col_join(J.T.row_join(sp.Matrix(H.tolist()).applyfunc(F)))
    gb = g0.col_join(sp.Matrix([F(v) for v in rt]))
    sol = Hb.LUsolve(-gb)
    x, u, y, dth = oracle.cross_stage_solve(prob, Jq, Jr, Jc, H, rt)
    dim = Hw.shape[0]
    exact_w = np.array([float(v) for v in sol[:dim]])
    np.testing.assert_allclose(oracle.join_solution(prob, x, u, y), exact_w, rtol=1e-10,
                               atol=1e-12)
    np.testing.assert_allclose(dth, [float(v) for v in sol[dim:]], rtol=1e-10, atol=1e-12)


def test_cross_stage_without_coupling_reduces_to_the_recursion():
    """J = 0 decouples the bordered system: dw is the LQR solution of the
    sequential recursion and dtheta = -H^{-1} r_theta."""
    prob = inputs.random_instance(31, 12, 3, 2, 1e-2)
    p_theta = 3
    rng = np.random.default_rng(31)
    H = rng.standard_normal((p_theta, p_theta))
    H = H @ H.T + np.eye(p_theta)
    rt = rng.standard_normal(p_theta)
    Z = lambda *s: np.zeros(s)  # noqa: E731
    x, u, y, dth = oracle.cross_stage_solve(prob, Z(p_theta, 13, 3), Z(p_theta, 12, 2),
                                            Z(p_theta, 13, 3), H, rt)
    ref = oracle.riccati(prob)
    np.testing.assert_allclose(x, ref.x, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(u, ref.u, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(y, ref.y, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(dth, -np.linalg.solve(H, rt), rtol=1e-12)
