"""Oracle for the regularized interior-point method on a nonlinear
multiple-shooting problem.  TEST INFRASTRUCTURE: only ``tests/``, the smoke
entry and the bench's CPU legs use it; it shares no code with the CUDA path.

What it computes, in the paper's notation (Section "The Regularized Interior
Point Method" and Section "Applying the regularized IPM to optimal control"):

  min f(x)  s.t.  c(x) = 0,  g(x) + s = 0,  s >= 0
  L(x, s, y, z; mu)  = f - mu sum log s + y^T c + z^T (g + s)
  A(x, s; y, z, mu)  = L + 1/2 (eta ||c||^2 + eta ||g + s||^2)     (merit)

Each iteration solves the Newton-KKT system eq. ipm-3x3-newton-kkt with
W = S Z^{-1}, Delta_C = Delta_G = eta I, by eliminating
Delta z = (W + Delta_G^{-1})^{-1} (G Delta x + r_z) and passing the reduced
(x, y) system to the dual-regularized LQR solve (delta = 1 / eta); then
Delta s = -W (Delta z - mu S^{-1} e + z).  The LQR step is the oracle's
sequential recursion (``oracle.riccati``), whose pivot-PD flags are the
inertia certificate: when a flag is not PD the Hessian is shifted by rho I
and the system re-solved within the same iteration (the rho I correction
after Theorem inertia-al-descent).  With correct inertia the primal direction descends the
merit function (Theorem inertia-al-descent), and a backtracking Armijo line
search on A with (y, z) fixed accepts the step.

Problem (a cart with a double pendulum; the paper names the task but does
not give its model, so the model is written out here from textbook
Lagrangian mechanics):
  state x = (p, th1, th2, dp, dth1, dth2): cart position, the two link
  angles from the upright (absolute), and their rates; control u = the
  horizontal force on the cart.  Point masses m1, m2 at the ends of massless
  links l1, l2, cart mass m0, gravity grav, no friction.
      M(th) qdd = tau(th, dth, u),  q = (p, th1, th2),
      M = [[m0+m1+m2, a1 cos th1, a2 cos th2],
           [a1 cos th1, b1, b12 cos(th1-th2)],
           [a2 cos th2, b12 cos(th1-th2), b2]]
      tau = (u + a1 sin th1 dth1^2 + a2 sin th2 dth2^2,
             a1 grav sin th1 - b12 sin(th1-th2) dth2^2,
             m2 grav l2 sin th2 + b12 sin(th1-th2) dth1^2)
  with a1 = (m1+m2) l1, a2 = m2 l2, b1 = (m1+m2) l1^2, b12 = m2 l1 l2,
  b2 = m2 l2^2.  Discretisation: classical RK4 with zero-order hold, step dt.
  Multiple shooting: c_0 = x0 - x_0, c_{i+1} = phi(x_i, u_i) - x_{i+1}.
  Cost: sum_{i<N} 1/2 (x_i-x_g)^T Wx (x_i-x_g) + 1/2 wu u_i^2
        + 1/2 (x_N-x_g)^T Wf (x_N-x_g), with diagonal Wx, Wf.
  Inequalities g <= 0 per stage: u - u_max, -u - u_max (i < N),
  p - p_max, -p - p_max (i = 0..N).

Constants the paper leaves open (this build's choices, the same on the GPU):
  Delta_C = Delta_G = eta I with eta = 1e3 (LQR delta = 1e-3); mu_0 = 0.1;
  mu <- max(mu_min, min(0.2 mu, mu^1.5)) once the barrier problem's KKT
  error E_mu <= 10 mu, mu_min = 1e-8; fraction to the boundary tau = 0.995
  for s and for z; Armijo constant 1e-4 with step halving from the
  fraction-to-boundary step of s, at most 12 trials (the last is taken if
  none passes), with an allowance of 10 eps |A| for rounding; y takes the
  primal step, z the smaller of its own fraction-to-boundary step and the
  primal step, then z is kept in [mu / (kappa s), kappa mu / s] with
  kappa = 1e10; rho (the inertia correction): every iteration first factors
  with a third of the last successful shift (0 if that was 0 or the third
  is below 1e-8); on a certificate failure a zero shift becomes 1e-4 (1e-8
  after a nonzero last shift) and a nonzero one grows x8, until every pivot
  is PD (failure above 1e8); convergence when
  max(||grad_x L||_inf, ||c||_inf, ||g + s||_inf, ||s z||_inf) <= 1e-6 (the
  benchmark tolerance of Section "Benchmarks"), at most 300 iterations;
  initial point: the rollout of the given controls (zeros for a cold start)
  or a given trajectory, y = 0, s = max(-g, 1e-2), z = mu_0 / s.
  The problem data (masses, lengths, dt, N, bounds, cost weights) are the
  workload's CDP_MODEL.

The Hessian of the Lagrangian is exact (the second derivatives of the RK4
map weighted by y), taken with second-order forward differentiation
(class ``Taylor2``); the Gauss-Newton variant drops that term.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from paper_2509_16370_b300.inputs import CDP_MODEL

from . import riccati

NX, NU, NW = 6, 1, 7
NG = 4                    # inequality rows per stage (0, 1: control; 2, 3: cart position)


# ---------------------------------------------------------------- parameters

@dataclass
class Model:
    """The problem data (defaults: the workload's CDP_MODEL)."""
    N: int = CDP_MODEL["N"]
    dt: float = CDP_MODEL["dt"]
    m0: float = CDP_MODEL["m0"]
    m1: float = CDP_MODEL["m1"]
    m2: float = CDP_MODEL["m2"]
    l1: float = CDP_MODEL["l1"]
    l2: float = CDP_MODEL["l2"]
    grav: float = CDP_MODEL["grav"]
    u_max: float = CDP_MODEL["u_max"]
    p_max: float = CDP_MODEL["p_max"]
    wx: tuple = CDP_MODEL["wx"]
    wu: float = CDP_MODEL["wu"]
    wf: tuple = CDP_MODEL["wf"]


@dataclass
class Options:
    max_iter: int = 300
    tol: float = 1e-6
    eta: float = 1e3
    mu0: float = 0.1
    mu_min: float = 1e-8
    kappa_mu: float = 10.0
    tau: float = 0.995
    armijo: float = 1e-4
    ls_steps: int = 12
    rho_first: float = 1e-4
    rho_grow: float = 8.0
    rho_shrink: float = 3.0
    rho_min: float = 1e-8
    rho_max: float = 1e8
    kappa_sigma: float = 1e10
    s_min: float = 1e-2
    exact_hessian: bool = True


# ------------------------------------------------ second-order forward mode

class Taylor2:
    """Value, gradient and Hessian of a function of NW variables, carried
    through +, -, *, /, sin, cos (vectorised over a leading stage axis)."""

    __slots__ = ("v", "g", "h")

    def __init__(self, v, g, h):
        self.v, self.g, self.h = v, g, h

    @staticmethod
    def variables(w):
        S = w.shape[0]
        out = []
        for k in range(w.shape[1]):
            g = np.zeros((S, w.shape[1]))
            g[:, k] = 1.0
            out.append(Taylor2(w[:, k].copy(), g, np.zeros((S, w.shape[1], w.shape[1]))))
        return out

    def _lift(self, o):
        if isinstance(o, Taylor2):
            return o
        o = np.broadcast_to(np.asarray(o, dtype=float), self.v.shape)
        return Taylor2(o, np.zeros_like(self.g), np.zeros_like(self.h))

    def __add__(self, o):
        o = self._lift(o)
        return Taylor2(self.v + o.v, self.g + o.g, self.h + o.h)

    __radd__ = __add__

    def __neg__(self):
        return Taylor2(-self.v, -self.g, -self.h)

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) - self

    def __mul__(self, o):
        if not isinstance(o, Taylor2):
            o = np.asarray(o, dtype=float)
            return Taylor2(self.v * o, self.g * o[..., None], self.h * o[..., None, None])
        gg = self.g[:, :, None] * o.g[:, None, :]
        return Taylor2(self.v * o.v, self.v[:, None] * o.g + o.v[:, None] * self.g,
                       self.v[:, None, None] * o.h + o.v[:, None, None] * self.h + gg
                       + np.swapaxes(gg, 1, 2))

    __rmul__ = __mul__

    def reciprocal(self):
        iv = 1.0 / self.v
        gg = self.g[:, :, None] * self.g[:, None, :]
        return Taylor2(iv, -self.g * (iv * iv)[:, None],
                       -self.h * (iv * iv)[:, None, None] + 2.0 * gg * (iv ** 3)[:, None, None])

    def __truediv__(self, o):
        if not isinstance(o, Taylor2):
            return self * (1.0 / np.asarray(o, dtype=float))
        return self * o.reciprocal()

    def sin(self):
        s, c = np.sin(self.v), np.cos(self.v)
        gg = self.g[:, :, None] * self.g[:, None, :]
        return Taylor2(s, c[:, None] * self.g, c[:, None, None] * self.h - s[:, None, None] * gg)

    def cos(self):
        s, c = np.sin(self.v), np.cos(self.v)
        gg = self.g[:, :, None] * self.g[:, None, :]
        return Taylor2(c, -s[:, None] * self.g, -s[:, None, None] * self.h - c[:, None, None] * gg)


def _sin(a):
    return a.sin() if isinstance(a, Taylor2) else np.sin(a)


def _cos(a):
    return a.cos() if isinstance(a, Taylor2) else np.cos(a)


# ------------------------------------------------------------------- model

def rhs(md: Model, x, u):
    """Continuous dynamics xdot = (dq, M^{-1} tau) for a list of six state
    components and the control (numbers, arrays, complex arrays or Taylor2)."""
    p, th1, th2, dp, w1, w2 = x
    a1 = (md.m1 + md.m2) * md.l1
    a2 = md.m2 * md.l2
    b1 = (md.m1 + md.m2) * md.l1 ** 2
    b12 = md.m2 * md.l1 * md.l2
    b2 = md.m2 * md.l2 ** 2
    mt = md.m0 + md.m1 + md.m2
    s1, c1, s2, c2 = _sin(th1), _cos(th1), _sin(th2), _cos(th2)
    s12, c12 = _sin(th1 - th2), _cos(th1 - th2)
    M11, M12, M13 = mt, a1 * c1, a2 * c2
    M22, M23, M33 = b1, b12 * c12, b2
    t1 = u + a1 * s1 * w1 * w1 + a2 * s2 * w2 * w2
    t2 = a1 * md.grav * s1 - b12 * s12 * w2 * w2
    t3 = md.m2 * md.grav * md.l2 * s2 + b12 * s12 * w1 * w1
    # M^{-1} tau by cofactors (M is symmetric positive definite)
    C11 = M22 * M33 - M23 * M23
    C12 = M13 * M23 - M12 * M33
    C13 = M12 * M23 - M13 * M22
    C22 = M11 * M33 - M13 * M13
    C23 = M12 * M13 - M11 * M23
    C33 = M11 * M22 - M12 * M12
    det = M11 * C11 + M12 * C12 + M13 * C13
    a_p = (C11 * t1 + C12 * t2 + C13 * t3) / det
    a_1 = (C12 * t1 + C22 * t2 + C23 * t3) / det
    a_2 = (C13 * t1 + C23 * t2 + C33 * t3) / det
    return [dp, w1, w2, a_p, a_1, a_2]


def rk4(md: Model, x, u):
    """One classical Runge-Kutta 4 step of length dt with the control held."""
    h = md.dt
    k1 = rhs(md, x, u)
    k2 = rhs(md, [a + 0.5 * h * b for a, b in zip(x, k1)], u)
    k3 = rhs(md, [a + 0.5 * h * b for a, b in zip(x, k2)], u)
    k4 = rhs(md, [a + h * b for a, b in zip(x, k3)], u)
    return [a + (h / 6.0) * (b1 + 2.0 * b2 + 2.0 * b3 + b4)
            for a, b1, b2, b3, b4 in zip(x, k1, k2, k3, k4)]


def step_map(md: Model, X, U):
    """phi(x_i, u_i) for stage-stacked X (S, 6), U (S,)."""
    out = rk4(md, [X[:, j] for j in range(NX)], U)
    return np.stack(out, axis=1)


def rollout(md: Model, x0, U):
    X = np.zeros((md.N + 1, NX))
    X[0] = x0
    for i in range(md.N):
        X[i + 1] = step_map(md, X[i:i + 1], U[i:i + 1])[0]
    return X


def energy(md: Model, x):
    """Total mechanical energy of the frictionless model (kinetic + potential)."""
    p, th1, th2, dp, w1, w2 = x
    v1x, v1y = dp + md.l1 * np.cos(th1) * w1, -md.l1 * np.sin(th1) * w1
    v2x = v1x + md.l2 * np.cos(th2) * w2
    v2y = v1y - md.l2 * np.sin(th2) * w2
    T = 0.5 * md.m0 * dp ** 2 + 0.5 * md.m1 * (v1x ** 2 + v1y ** 2) + \
        0.5 * md.m2 * (v2x ** 2 + v2y ** 2)
    V = md.m1 * md.grav * md.l1 * np.cos(th1) + \
        md.m2 * md.grav * (md.l1 * np.cos(th1) + md.l2 * np.cos(th2))
    return T + V


def linearize_dynamics(md: Model, X, U, Y):
    """Per stage i < N: phi_i (N, 6), A_i (N, 6, 6), B_i (N, 6, 1) and the
    Hessian of y_{i+1}^T phi(x_i, u_i) in (x_i, u_i) (N, 7, 7)."""
    N = md.N
    w = np.concatenate([X[:N], U[:, None]], axis=1)
    v = Taylor2.variables(w)
    phi = rk4(md, v[:NX], v[NX])
    val = np.stack([t.v for t in phi], axis=1)
    jac = np.stack([t.g for t in phi], axis=1)              # (N, 6, 7)
    hy = sum(Y[1:, l][:, None, None] * phi[l].h for l in range(NX))
    return val, jac[:, :, :NX], jac[:, :, NX:], hy


# ------------------------------------------------------------ IPM pieces

def inequalities(md: Model, X, U):
    """g (N+1, 4) and the mask of existing rows (the control rows at i = N
    do not exist)."""
    N = md.N
    g = np.zeros((N + 1, NG))
    g[:N, 0] = U - md.u_max
    g[:N, 1] = -U - md.u_max
    g[:, 2] = X[:, 0] - md.p_max
    g[:, 3] = -X[:, 0] - md.p_max
    mask = np.ones((N + 1, NG), dtype=bool)
    mask[N, :2] = False
    return g, mask


def cost(md: Model, X, U, xg):
    d = X - xg
    wx, wf = np.asarray(md.wx), np.asarray(md.wf)
    return 0.5 * np.sum(d[:-1] ** 2 * wx) + 0.5 * md.wu * np.sum(U ** 2) + \
        0.5 * np.sum(d[-1] ** 2 * wf)


def defects(md: Model, x0, X, U, phi=None):
    """c_0 = x0 - x_0, c_{i+1} = phi(x_i, u_i) - x_{i+1}  (N+1, 6)."""
    if phi is None:
        phi = step_map(md, X[:-1], U)
    c = np.empty_like(X)
    c[0] = x0 - X[0]
    c[1:] = phi - X[1:]
    return c


def merit(md: Model, op: Options, st, X, U, S, mu):
    """Augmented barrier-Lagrangian A(x, s; y, z, mu) at (X, U, S) with the
    iterate's duals (the merit of the line search)."""
    g, mask = inequalities(md, X, U)
    c = defects(md, st.x0, X, U)
    gs = (g + S)[mask]
    return (cost(md, X, U, st.xg) - mu * np.sum(np.log(S[mask])) + np.sum(st.Y * c)
            + np.sum(st.Z[mask] * gs) + 0.5 * op.eta * np.sum(c * c)
            + 0.5 * op.eta * np.sum(gs * gs))


@dataclass
class State:
    x0: np.ndarray
    xg: np.ndarray
    X: np.ndarray
    U: np.ndarray
    Y: np.ndarray
    S: np.ndarray
    Z: np.ndarray
    mu: float
    rho: float = 0.0          # last shift that gave the correct inertia
    iters: int = 0
    factorizations: int = 0
    status: int = 0          # 0 running, 1 converged, 2 iteration limit, 3 rho limit
    history: list = field(default_factory=list)

    def copy(self):
        return State(self.x0.copy(), self.xg.copy(), self.X.copy(), self.U.copy(),
                     self.Y.copy(), self.S.copy(), self.Z.copy(), self.mu, self.rho,
                     self.iters, self.factorizations, self.status, list(self.history))


def initial_state(md: Model, op: Options, x0, xg, U=None, X=None):
    """Initial point: the rollout of U (zeros if None) unless X is given;
    y = 0, s = max(-g, s_min), z = mu_0 / s (1 on rows that do not exist)."""
    U = np.zeros(md.N) if U is None else np.asarray(U, dtype=float).copy()
    X = rollout(md, x0, U) if X is None else np.asarray(X, dtype=float).copy()
    g, mask = inequalities(md, X, U)
    S = np.where(mask, np.maximum(-g, op.s_min), 1.0)
    Z = np.where(mask, op.mu0 / S, 0.0)
    return State(np.asarray(x0, float).copy(), np.asarray(xg, float).copy(), X, U,
                 np.zeros_like(X), S, Z, op.mu0)


@dataclass
class Linearization:
    phi: np.ndarray
    A: np.ndarray
    B: np.ndarray
    H: np.ndarray           # (N, 7, 7) Hessian of the dynamics term (0 for Gauss-Newton)
    c: np.ndarray           # (N+1, 6) defects
    gx: np.ndarray          # (N+1, 6) grad_x L
    gu: np.ndarray          # (N,) grad_u L
    g: np.ndarray           # (N+1, 4) inequality values
    mask: np.ndarray
    err0: float             # max(||grad L||, ||c||, ||g + s||, ||s z||)
    err_mu: float           # the same with ||s z - mu||


def linearize(md: Model, op: Options, st: State) -> Linearization:
    N = md.N
    phi, A, B, H = linearize_dynamics(md, st.X, st.U, st.Y)
    if not op.exact_hessian:
        H = np.zeros_like(H)
    c = defects(md, st.x0, st.X, st.U, phi)
    g, mask = inequalities(md, st.X, st.U)
    wx, wf = np.asarray(md.wx), np.asarray(md.wf)
    d = st.X - st.xg
    gx = np.empty_like(st.X)
    gx[:N] = d[:N] * wx + np.einsum("ilj,il->ij", A, st.Y[1:]) - st.Y[:N]
    gx[N] = d[N] * wf - st.Y[N]
    gx[:, 0] += st.Z[:, 2] - st.Z[:, 3]
    gu = md.wu * st.U + np.einsum("il,il->i", B[:, :, 0], st.Y[1:]) + st.Z[:N, 0] - st.Z[:N, 1]
    gs = np.abs((g + st.S)[mask])
    sz = (st.S * st.Z)[mask]
    base = max(np.abs(gx).max(), np.abs(gu).max(), np.abs(c).max(), gs.max())
    return Linearization(phi, A, B, H, c, gx, gu, g, mask, max(base, np.abs(sz).max()),
                         max(base, np.abs(sz - st.mu).max()))


class _LQR:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def newton_lqr(md: Model, op: Options, st: State, lin: Linearization, rho: float):
    """The reduced Newton system as a dual-regularized LQR (Section
    "Applying the regularized IPM to optimal control"), its certificate and
    its solution mapped back to (dx, du, ds, dy, dz)."""
    N, mu = md.N, st.mu
    m = lin.mask
    Dg = np.where(m, 1.0 / (st.S / np.where(m, st.Z, 1.0) + 1.0 / op.eta), 0.0)
    rz = np.where(m, lin.g + mu / np.where(m, st.Z, 1.0), 0.0)
    Q = np.zeros((N + 1, NX, NX))
    Q[:N] = lin.H[:, :NX, :NX]
    Q[:N] += np.diag(md.wx)
    Q[N] += np.diag(md.wf)
    Q += rho * np.eye(NX)
    Q[:, 0, 0] += Dg[:, 2] + Dg[:, 3]
    Mx = lin.H[:, :NX, NX:].copy()
    R = lin.H[:, NX:, NX:].copy() + md.wu + rho
    R[:, 0, 0] += Dg[:N, 0] + Dg[:N, 1]
    q = lin.gx.copy()
    q[:, 0] += Dg[:, 2] * rz[:, 2] - Dg[:, 3] * rz[:, 3]
    r = (lin.gu + Dg[:N, 0] * rz[:N, 0] - Dg[:N, 1] * rz[:N, 1])[:, None]
    prob = _LQR(N=N, n=NX, m=NU, Q=Q, M=Mx, R=R, q=q, r=r, A=lin.A, B=lin.B, c=lin.c,
                delta=1.0 / op.eta)
    res = riccati(prob)
    dX, dU, dY = res.x, res.u[:, 0], res.y
    Gdx = np.zeros((N + 1, NG))
    Gdx[:N, 0], Gdx[:N, 1] = dU, -dU
    Gdx[:, 2], Gdx[:, 3] = dX[:, 0], -dX[:, 0]
    dZ = np.where(m, Dg * (Gdx + rz), 0.0)
    W = np.where(m, st.S / np.where(m, st.Z, 1.0), 0.0)
    dS = np.where(m, -W * dZ + mu / np.where(m, st.Z, 1.0) - st.S, 0.0)
    return res, prob, dX, dU, dS, dY, dZ, Gdx


def fraction_to_boundary(v, dv, mask, tau):
    neg = mask & (dv < 0)
    if not neg.any():
        return 1.0
    return float(min(1.0, np.min(-tau * v[neg] / dv[neg])))


def merit_slope(md: Model, op: Options, st: State, lin: Linearization, dX, dU, dS, Gdx):
    """Directional derivative of the merit along (dx, ds) with (y, z) fixed:
    grad f . dx + (y + eta c)^T C dx + (z + eta_g (g + s))^T (G dx + ds)
    - mu sum ds / s."""
    N = md.N
    m = lin.mask
    d = st.X - st.xg
    gf = np.sum(d[:N] * np.asarray(md.wx) * dX[:N]) + np.sum(d[N] * np.asarray(md.wf) * dX[N]) \
        + md.wu * np.sum(st.U * dU)
    Cdx = np.empty_like(dX)
    Cdx[0] = -dX[0]
    Cdx[1:] = np.einsum("ijk,ik->ij", lin.A, dX[:N]) + lin.B[:, :, 0] * dU[:, None] - dX[1:]
    lam = st.Y + op.eta * lin.c
    nu = st.Z + op.eta * (lin.g + st.S)
    return gf + np.sum(lam * Cdx) + np.sum((nu * (Gdx + dS))[m]) - st.mu * np.sum((dS / st.S)[m])


def iterate(md: Model, op: Options, st: State) -> State:
    """One iteration (one Newton system) on a running instance, in place."""
    lin = linearize(md, op, st)
    if lin.err0 <= op.tol:
        st.status = 1
        return st
    if st.iters >= op.max_iter:
        st.status = 2
        return st
    if lin.err_mu <= op.kappa_mu * st.mu:
        st.mu = max(op.mu_min, min(0.2 * st.mu, st.mu ** 1.5))
    st.iters += 1
    # inertia correction: the first try is a third of the last shift that
    # gave the correct inertia (0 if that was 0 or the third is below
    # rho_min); on a certificate failure a zero shift becomes rho_first (or
    # rho_min after a nonzero last shift) and a nonzero one grows x8, until
    # every pivot is PD
    rho = st.rho / op.rho_shrink if st.rho / op.rho_shrink > op.rho_min else 0.0
    while True:
        res, prob, dX, dU, dS, dY, dZ, Gdx = newton_lqr(md, op, st, lin, rho)
        st.factorizations += 1
        if res.status < 2 and bool(np.all(res.flags == 3)):
            break
        if rho == 0.0:
            rho = op.rho_first if st.rho == 0.0 else max(op.rho_min, st.rho / op.rho_shrink)
        else:
            rho *= op.rho_grow
        if rho > op.rho_max:
            st.status = 3
            st.history.append(dict(it=st.iters, mu=st.mu, rho=rho, err0=lin.err0, alpha=0.0))
            return st
    st.rho = rho
    rec = dict(it=st.iters, mu=st.mu, rho=rho, err0=lin.err0, alpha=0.0, trials=0)
    st.history.append(rec)
    m = lin.mask
    a_s = fraction_to_boundary(st.S, dS, m, op.tau)
    a_z = fraction_to_boundary(st.Z, dZ, m, op.tau)
    A0 = merit(md, op, st, st.X, st.U, st.S, st.mu)
    slope = merit_slope(md, op, st, lin, dX, dU, dS, Gdx)
    allowance = 10.0 * np.finfo(float).eps * abs(A0)
    for k in range(op.ls_steps):
        alpha = a_s * 0.5 ** k
        Sn = np.where(m, st.S + alpha * dS, 1.0)
        At = merit(md, op, st, st.X + alpha * dX, st.U + alpha * dU, Sn, st.mu)
        if At <= A0 + op.armijo * alpha * slope + allowance:
            break
    rec.update(alpha=alpha, trials=k + 1, slope=slope, merit=A0)
    st.X = st.X + alpha * dX
    st.U = st.U + alpha * dU
    st.S = np.where(m, st.S + alpha * dS, 1.0)
    st.Y = st.Y + alpha * dY
    # the bound duals take at most the primal step, then are kept within a
    # factor kappa_sigma of mu / s
    a_z = min(a_z, alpha)
    Sm = np.where(m, st.S, 1.0)
    st.Z = np.where(m, np.clip(st.Z + a_z * dZ, st.mu / (op.kappa_sigma * Sm),
                               op.kappa_sigma * st.mu / Sm), 0.0)
    return st


def solve(md: Model, op: Options, x0, xg, U=None, X=None) -> State:
    st = initial_state(md, op, x0, xg, U, X)
    while st.status == 0:
        iterate(md, op, st)
    return st


def kkt_error(md: Model, op: Options, st: State) -> float:
    """max(||grad_x L||, ||c||, ||g + s||, ||s z||) at the state (mu = 0)."""
    return linearize(md, op, st).err0


# ------------------------------------------------------- dense Newton step

def newton_dense(md: Model, op: Options, st: State, lin: Linearization, rho: float):
    """The full Newton-KKT system eq. ipm-4x4-newton-kkt, assembled densely
    over (x, s, y, z) and solved by numpy: the plain definition that the
    LQR route must reproduce (small N only)."""
    N = md.N
    m = lin.mask
    nxu = N * (NX + NU) + NX
    rows = np.argwhere(m)                       # existing inequality rows (i, k)
    ng, nc = len(rows), (N + 1) * NX

    def xi(i):
        return i * (NX + NU)

    P = np.zeros((nxu, nxu))
    gradx = np.zeros(nxu)
    for i in range(N):
        o = xi(i)
        P[o:o + NW, o:o + NW] = lin.H[i]
        P[o:o + NX, o:o + NX] += np.diag(md.wx)
        P[o + NX, o + NX] += md.wu
        gradx[o:o + NX] = lin.gx[i]
        gradx[o + NX] = lin.gu[i]
    P[xi(N):, xi(N):] += np.diag(md.wf)
    gradx[xi(N):] = lin.gx[N]
    P += rho * np.eye(nxu)
    C = np.zeros((nc, nxu))
    C[0:NX, 0:NX] = -np.eye(NX)
    for i in range(N):
        r0 = (i + 1) * NX
        C[r0:r0 + NX, xi(i):xi(i) + NX] = lin.A[i]
        C[r0:r0 + NX, xi(i) + NX] = lin.B[i][:, 0]
        C[r0:r0 + NX, xi(i + 1):xi(i + 1) + NX] = -np.eye(NX)
    G = np.zeros((ng, nxu))
    for r, (i, k) in enumerate(rows):
        sign = 1.0 if k % 2 == 0 else -1.0
        G[r, xi(i) + (NX if k < 2 else 0)] = sign
    s = st.S[m]
    z = st.Z[m]
    g = lin.g[m]
    dim = nxu + ng + nc + ng
    K = np.zeros((dim, dim))
    o1, o2, o3 = nxu, nxu + ng, nxu + ng + nc
    K[:nxu, :nxu] = P
    K[:nxu, o2:o3] = C.T
    K[:nxu, o3:] = G.T
    K[o1:o2, o1:o2] = np.diag(z / s)            # W^{-1}
    K[o1:o2, o3:] = np.eye(ng)
    K[o2:o3, :nxu] = C
    K[o2:o3, o2:o3] = -np.eye(nc) / op.eta
    K[o3:, :nxu] = G
    K[o3:, o1:o2] = np.eye(ng)
    K[o3:, o3:] = -np.eye(ng) / op.eta
    rhs_ = -np.concatenate([gradx, -st.mu / s + z, lin.c.ravel(), g + s])
    sol = np.linalg.solve(K, rhs_)
    dx = sol[:nxu]
    dX = np.zeros((N + 1, NX))
    dU = np.zeros(N)
    for i in range(N):
        dX[i] = dx[xi(i):xi(i) + NX]
        dU[i] = dx[xi(i) + NX]
    dX[N] = dx[xi(N):]
    dS = np.zeros((N + 1, NG))
    dZ = np.zeros((N + 1, NG))
    dS[m] = sol[o1:o2]
    dZ[m] = sol[o3:]
    dY = sol[o2:o3].reshape(N + 1, NX)
    return dict(dX=dX, dU=dU, dS=dS, dY=dY, dZ=dZ, K=K, rhs=rhs_, P=P, C=C, G=G)
