"""Seeded synthetic inputs for the dual-regularized LQR solver.

This module holds the input recipes only: it draws random problem data and
does none of the method's arithmetic (no Riccati step, no pivot, no solve).
Both the CUDA path (tests, bench) and the CPU oracle take their inputs from
here.  Pivot margins, which do need the method, are decided by a script that
calls only the oracle (``tests/golden/make_curation.py``); its output table
(``tests/golden/workload2_curation.json``) is read here as plain data.

Data layout (one instance): stage-major, row-major FP64 arrays
  Q (N+1, n, n)  M (N, n, m)  R (N, m, m)  q (N+1, n)  r (N, m)
  A (N, n, n)    B (N, n, m)  c (N+1, n)   and a scalar delta (Delta_i = delta I).
A uniform batch stacks these along a leading instance axis (delta per instance).

Seeds: numpy PCG64 seeded from SeedSequence([20250916, workload, instance, sub]),
where ``sub`` counts redraws of an instance.

Recipes (shapes of the paper's trajectory-optimisation problems, see the
benchmark table of Section "Benchmarks"):
  * "Gaussian rescaled to spectral radius rho": A_i = G rho / max|eig(G)|,
    drawn independently per stage.
  * "LL^T + eps I": L with N(0,1) entries.
  * "condition number kappa": U diag(logspace(0, -log10 kappa, n)) U^T with U
    from the QR of a Gaussian (spectral norm 1).

Workloads
  1  single instance, n=4, m=2, N=64, delta=1e-6, rho(A)=0.95, B,c,q,r ~ N(0,1),
     Q = LL^T + 1e-2 I (all N+1), R = KK^T + 1e-2 I, M = 0.
  2  1024 instances, n=12, m=4, N=256, delta = 10^U(-8,-2) per instance, base as
     workload 1; instances with index mod 10 in {0,1,2} have every Q_i with two
     eigenvalues in -U(0.01, 0.1) and the rest in U(0.5, 2) (non-convex Hessian);
     index mod 20 == 7 is made pivot-indefinite on purpose at one stage k* by
     lowering R_{k*} by alpha I (k*, alpha from the curation table).
  3  single instance, n=32, m=8, N=65536, delta=1e-7, rho(A)=0.99, Q and R with
     condition number 1e4, M = 0.
  4  ragged batch of 4096: N ~ U{32..2048}, n ~ U{6,12,24,48}, m = n/3, base as
     workload 1 plus M = 0.1 N(0,1), delta = 10^U(-8,-2), and a barrier term
     10^U(-6,6) added to every diagonal entry of Q_i and R_i.
  5  8192 cart-double-pendulum trajectory problems (CDP_MODEL): initial state
     at rest at p = 0 with both link angles uniform in [-pi, pi], goal state
     (p_goal, 0, 0, 0, 0, 0) with p_goal uniform in [-1, 1].
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20250916
_HERE = os.path.dirname(os.path.abspath(__file__))
CURATION_PATH = os.path.join(os.path.dirname(_HERE), "tests", "golden", "workload2_curation.json")


@dataclass
class Problem:
    """One dual-regularized LQR instance (FP64, stage-major)."""
    N: int
    n: int
    m: int
    Q: np.ndarray
    M: np.ndarray
    R: np.ndarray
    q: np.ndarray
    r: np.ndarray
    A: np.ndarray
    B: np.ndarray
    c: np.ndarray
    delta: float
    meta: dict = field(default_factory=dict)

    def arrays(self):
        return dict(Q=self.Q, M=self.M, R=self.R, q=self.q, r=self.r, A=self.A, B=self.B,
                    c=self.c)


@dataclass
class Batch:
    """``count`` instances of equal (N, n, m) stacked along axis 0."""
    count: int
    N: int
    n: int
    m: int
    Q: np.ndarray
    M: np.ndarray
    R: np.ndarray
    q: np.ndarray
    r: np.ndarray
    A: np.ndarray
    B: np.ndarray
    c: np.ndarray
    delta: np.ndarray
    meta: list = field(default_factory=list)

    def instance(self, b: int) -> Problem:
        return Problem(self.N, self.n, self.m, self.Q[b], self.M[b], self.R[b], self.q[b],
                       self.r[b], self.A[b], self.B[b], self.c[b], float(self.delta[b]),
                       self.meta[b] if self.meta else {})

    @staticmethod
    def stack(probs):
        p0 = probs[0]
        assert all((p.N, p.n, p.m) == (p0.N, p0.n, p0.m) for p in probs)
        st = {k: np.ascontiguousarray(np.stack([getattr(p, k) for p in probs]))
              for k in ("Q", "M", "R", "q", "r", "A", "B", "c")}
        return Batch(len(probs), p0.N, p0.n, p0.m, delta=np.array([p.delta for p in probs]),
                     meta=[p.meta for p in probs], **st)


def rng_for(workload: int, instance: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(
        [SEED_BASE, int(workload), int(instance), int(sub)])))


# ------------------------------------------------------------------ recipes

def spectral_rescaled(rng, count: int, n: int, rho: float) -> np.ndarray:
    """``count`` Gaussian n x n matrices, each rescaled to spectral radius rho."""
    G = rng.standard_normal((count, n, n))
    rad = np.abs(np.linalg.eigvals(G)).max(axis=-1)
    return G * (rho / rad)[:, None, None]


def llt_plus(rng, count: int, n: int, eps: float) -> np.ndarray:
    """``count`` matrices L L^T + eps I with L ~ N(0,1) (exactly symmetric)."""
    L = rng.standard_normal((count, n, n))
    X = L @ np.swapaxes(L, -1, -2) + eps * np.eye(n)
    return 0.5 * (X + np.swapaxes(X, -1, -2))


def orthogonal(rng, count: int, n: int) -> np.ndarray:
    Qm, Rm = np.linalg.qr(rng.standard_normal((count, n, n)))
    return Qm * np.sign(np.diagonal(Rm, axis1=-2, axis2=-1))[:, None, :]


def with_spectrum(U: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """U diag(lam) U^T, batched, exactly symmetric."""
    X = (U * lam[:, None, :]) @ np.swapaxes(U, -1, -2)
    return 0.5 * (X + np.swapaxes(X, -1, -2))


def cond_spd(rng, count: int, n: int, kappa: float) -> np.ndarray:
    """SPD matrices with eigenvalues logspace(0, -log10 kappa, n) (norm 1)."""
    lam = np.broadcast_to(np.logspace(0.0, -np.log10(kappa), n), (count, n))
    return with_spectrum(orthogonal(rng, count, n), lam)


def base_instance(rng, N, n, m, delta, rho=0.95, eps=1e-2) -> Problem:
    """The common recipe: A_i Gaussian at spectral radius rho, B, c, q, r ~ N(0,1),
    Q_i = LL^T + eps I, R_i = KK^T + eps I, M = 0."""
    A = spectral_rescaled(rng, N, n, rho)
    B = rng.standard_normal((N, n, m))
    c = rng.standard_normal((N + 1, n))
    q = rng.standard_normal((N + 1, n))
    r = rng.standard_normal((N, m))
    Q = llt_plus(rng, N + 1, n, eps)
    R = llt_plus(rng, N, m, eps)
    M = np.zeros((N, n, m))
    return Problem(N, n, m, Q, M, R, q, r, A, B, c, float(delta))


# ---------------------------------------------------------------- workloads

def workload1() -> Problem:
    """Single instance, n=4, m=2, N=64, delta=1e-6."""
    p = base_instance(rng_for(1, 0), 64, 4, 2, 1e-6)
    p.meta = dict(workload=1, instance=0)
    return p


def _load_curation():
    if not os.path.exists(CURATION_PATH):
        return None
    with open(CURATION_PATH) as f:
        return json.load(f)


def workload2_kind(b: int) -> str:
    if b % 20 == 7:
        return "indefinite"
    if b % 10 in (0, 1, 2):
        return "nonconvex"
    return "convex"


def workload2_instance(b: int, N: int = 256, n: int = 12, m: int = 4, sub: int = 0,
                       kstar: int | None = None, alpha: float = 0.0) -> Problem:
    """Instance ``b`` of workload 2 for redraw ``sub``; an indefinite instance
    gets R_{kstar} -= alpha I."""
    rng = rng_for(2, b, sub)
    delta = 10.0 ** rng.uniform(-8.0, -2.0)
    p = base_instance(rng, N, n, m, delta)
    kind = workload2_kind(b)
    if kind == "nonconvex":
        lam = np.empty((N + 1, n))
        lam[:, :2] = -rng.uniform(0.01, 0.1, size=(N + 1, 2))
        lam[:, 2:] = rng.uniform(0.5, 2.0, size=(N + 1, n - 2))
        p.Q = with_spectrum(orthogonal(rng, N + 1, n), lam)
    if kind == "indefinite" and kstar is not None:
        p.R = p.R.copy()
        p.R[kstar] -= alpha * np.eye(m)
    p.meta = dict(workload=2, instance=b, kind=kind, sub=sub, kstar=kstar, alpha=alpha)
    return p


def workload2(count: int = 1024, N: int = 256, n: int = 12, m: int = 4,
              curation=None, require_curation: bool = True) -> Batch:
    """Batch of ``count`` instances (n=12, m=4, N=256 by default).

    The redraw index and the indefinite-pivot shift of each instance come from
    the curation table when it matches these sizes."""
    if curation is None:
        curation = _load_curation()
    key = f"N{N}_n{n}_m{m}"
    table = None
    if curation is not None and key in curation.get("tables", {}):
        table = curation["tables"][key]
    if table is None and require_curation:
        raise FileNotFoundError(f"no curation table for {key} in {CURATION_PATH}")
    probs = []
    for b in range(count):
        ent = table[str(b)] if table is not None and str(b) in table else {}
        probs.append(workload2_instance(b, N, n, m, sub=ent.get("sub", 0),
                                        kstar=ent.get("kstar"), alpha=ent.get("alpha", 0.0)))
    return Batch.stack(probs)


def workload3(N: int = 65536, n: int = 32, m: int = 8) -> Problem:
    """Single long-horizon instance: n=32, m=8, N=65536, delta=1e-7,
    rho(A)=0.99, Q_i and R_i with condition number 1e4, M = 0."""
    rng = rng_for(3, 0)
    A = spectral_rescaled(rng, N, n, 0.99)
    B = rng.standard_normal((N, n, m))
    c = rng.standard_normal((N + 1, n))
    q = rng.standard_normal((N + 1, n))
    r = rng.standard_normal((N, m))
    Q = cond_spd(rng, N + 1, n, 1e4)
    R = cond_spd(rng, N, m, 1e4)
    M = np.zeros((N, n, m))
    return Problem(N, n, m, Q, M, R, q, r, A, B, c, 1e-7, dict(workload=3, instance=0))


def workload4_dims(count: int = 4096):
    """(N, n, m) of each instance of the ragged workload 4."""
    rng = rng_for(4, 1 << 30)
    Ns = rng.integers(32, 2049, size=count)
    ns = rng.choice(np.array([6, 12, 24, 48]), size=count)
    return [(int(a), int(b), int(b) // 3) for a, b in zip(Ns, ns)]


def workload4_instance(b: int, N: int, n: int, m: int) -> Problem:
    rng = rng_for(4, b)
    delta = 10.0 ** rng.uniform(-8.0, -2.0)
    p = base_instance(rng, N, n, m, delta)
    p.M = 0.1 * rng.standard_normal((N, n, m))
    idx_n = np.arange(n)
    idx_m = np.arange(m)
    p.Q[:, idx_n, idx_n] += 10.0 ** rng.uniform(-6.0, 6.0, size=(N + 1, n))
    p.R[:, idx_m, idx_m] += 10.0 ** rng.uniform(-6.0, 6.0, size=(N, m))
    p.meta = dict(workload=4, instance=b)
    return p


def random_instance(seed: int, N: int, n: int, m: int, delta: float, with_M: bool = True,
                    rho: float = 0.95) -> Problem:
    """Small generic instance for unit tests (M ~ 0.3 N(0,1) when with_M)."""
    rng = rng_for(99, seed)
    p = base_instance(rng, N, n, m, delta, rho=rho)
    if with_M:
        p.M = 0.3 * rng.standard_normal((N, n, m))
    p.meta = dict(workload=99, instance=seed)
    return p


# The cart-double-pendulum problem of workload 5 (plain data: masses in kg,
# lengths in m, the RK4 step dt in s, N steps, bounds, diagonal cost weights;
# the stage weights are per step, i.e. the continuous weights times dt).
CDP_MODEL = dict(N=128, dt=0.02, m0=1.0, m1=0.5, m2=0.5, l1=0.5, l2=0.5, grav=9.81,
                 u_max=20.0, p_max=2.0, wx=(0.02, 0.02, 0.02, 0.002, 0.002, 0.002),
                 wu=2e-4, wf=(10.0, 10.0, 10.0, 1.0, 1.0, 1.0))


def workload5_instance(b: int):
    """Initial state and goal of instance b of the cart-double-pendulum batch
    (8192 instances): cart at rest at p = 0, both link angles uniform in
    [-pi, pi] from the upright, rates zero; goal state (p_goal, 0, 0, 0, 0, 0)
    with p_goal uniform in [-1, 1]."""
    rng = rng_for(5, b)
    th = rng.uniform(-np.pi, np.pi, size=2)
    pg = rng.uniform(-1.0, 1.0)
    x0 = np.array([0.0, th[0], th[1], 0.0, 0.0, 0.0])
    xg = np.array([pg, 0.0, 0.0, 0.0, 0.0, 0.0])
    return x0, xg


def workload5(count: int = 8192, start: int = 0):
    """Stacked initial states (count, 6) and goals (count, 6) of instances
    start .. start + count - 1."""
    x0 = np.zeros((count, 6))
    xg = np.zeros((count, 6))
    for b in range(count):
        x0[b], xg[b] = workload5_instance(start + b)
    return x0, xg
