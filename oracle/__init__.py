"""FP64 CPU oracle for the dual-regularized LQR solve.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and the library never calls
it.  Everything here is plain FP64: the C file ``rlqr_oracle.c`` for the loops
and numpy for the dense assembly of the KKT matrix.

What it computes (citations are to the paper's sections and equations):

* ``riccati``      -- the sequential dual-regularized Riccati recursion of
  Section "Sequential Algorithm" (Theorem main-seq-theorem, eq.
  value-fn-formulas, control-law, recover-x0, recover-x) with the pivot-PD
  certificate of Section "Inertia Certification".
* ``kkt_dense``    -- the matrix and right-hand side of eq.
  primal-dual-linear-system with the blocks of eq.
  optimal-control-specialization.
* ``dense_solve``  -- Bunch-Kaufman LDL^T of that matrix: the unique solution
  and the inertia from D (the plain definition of what the method computes).
* ``jacobi_inertia`` -- eigenvalue inertia count by cyclic Jacobi.
* ``band_solve``   -- the same system solved by banded LU with partial
  pivoting in the interleaved order (for sizes where a dense factor is too big).
* ``residual``     -- the stagewise residual of Section "Residual Computation"
  and the normwise backward error.
* ``kkt_dense_diag`` / ``riccati_diag`` -- a general diagonal Delta_i
  (Section "Dual-Regularized LQR" allows any SPD Delta_i): the dense system
  and the recursion with S_i = I + Delta_i^{1/2} P_i Delta_i^{1/2}.
* ``cross_stage_solve`` -- Section "Cross-Stage Variables": the bordered
  system [[K, J], [J^T, H]] [dw; dtheta] = -[b; r_theta], assembled densely
  from ``kkt_dense`` and solved by numpy (the plain definition).

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: the paper's two worked examples, exact rational solves of the
Lagrangian's stationarity conditions, the scalar steady-state closed form,
scipy's discrete algebraic Riccati equation at delta = 0, numpy's eigvalsh
inertia, and the inertia identity of Theorem
riccati-inertia-certification-theorem.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlqr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

OK, NOT_PD, ERR_ARG, SINGULAR = 0, 1, 2, 3

# -O3 -march=native for the timed CPU baseline; -ffp-contract=off keeps every
# operation a separately rounded FP64 operation in the source's order (no
# fused multiply-adds, no reassociation), as in a plain evaluation.
CFLAGS = ["-O3", "-march=native", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared",
          "-fopenmp"]


def _cpu_tag() -> str:
    """A tag of the host CPU (model and feature flags): -march=native code is
    built per CPU, so a library built on another machine is never loaded."""
    import hashlib
    try:
        with open("/proc/cpuinfo") as f:
            info = [ln for ln in f if ln.startswith(("model name", "flags"))][:2]
    except OSError:
        info = []
    return hashlib.sha1("".join(info).encode()).hexdigest()[:12]


_LIB_PATH = os.path.join(_BUILD, f"librlqr_oracle.{_cpu_tag()}.so")


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (CFLAGS, OpenMP over instances)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc"] + CFLAGS + ["-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i32, u8, i = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                         ctypes.POINTER(ctypes.c_uint8), ctypes.c_int)
        lib.rlqr_orc_riccati.restype = ctypes.c_int
        lib.rlqr_orc_riccati.argtypes = [i, i, i] + [d] * 8 + [ctypes.c_double] + [d] * 3 + [
            u8, i32, i32] + [d] * 6
        lib.rlqr_orc_riccati_batch.restype = None
        lib.rlqr_orc_riccati_batch.argtypes = [i, i, i, i] + [d] * 9 + [d] * 3 + [u8, i32]
        lib.rlqr_orc_bk_factor.restype = ctypes.c_int
        lib.rlqr_orc_bk_factor.argtypes = [i, d, i32, i32]
        lib.rlqr_orc_bk_solve.restype = None
        lib.rlqr_orc_bk_solve.argtypes = [i, d, i32, i32, d]
        lib.rlqr_orc_bk_inertia.restype = None
        lib.rlqr_orc_bk_inertia.argtypes = [i, d, i32, i32]
        lib.rlqr_orc_jacobi_inertia.restype = ctypes.c_int
        lib.rlqr_orc_jacobi_inertia.argtypes = [i, d, ctypes.c_double, i, i32, d]
        lib.rlqr_orc_band_solve.restype = ctypes.c_int
        lib.rlqr_orc_band_solve.argtypes = [i, i, i] + [d] * 8 + [ctypes.c_double] + [d] * 3
        lib.rlqr_orc_residual.restype = None
        lib.rlqr_orc_residual.argtypes = [i, i, i] + [d] * 8 + [ctypes.c_double] + [d] * 3 + [
            d] * 4
        _lib = lib
    return _lib


def _p(a, ctype=ctypes.c_double):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _data(prob):
    return [_f64(getattr(prob, k)) for k in ("Q", "M", "R", "q", "r", "A", "B", "c")]


@dataclass
class RiccatiResult:
    status: int
    x: np.ndarray
    u: np.ndarray
    y: np.ndarray
    flags: np.ndarray
    neg_S: np.ndarray | None = None
    neg_G: np.ndarray | None = None
    P: np.ndarray | None = None
    p: np.ndarray | None = None
    K: np.ndarray | None = None
    k: np.ndarray | None = None
    S: np.ndarray | None = None
    G: np.ndarray | None = None


def riccati(prob, internals: bool = False) -> RiccatiResult:
    """Sequential recursion (Section "Sequential Algorithm") on one instance.

    ``prob`` has fields N, n, m, Q, M, R, q, r, A, B, c (stage-major FP64
    arrays, shapes (N+1,n,n), (N,n,m), (N,m,m), (N+1,n), (N,m), (N,n,n),
    (N,n,m), (N+1,n)) and delta.  ``flags[i]`` bit0: I + delta P_i is PD;
    bit1: G_i is PD (set at i = N).  With ``internals`` it also returns the
    negative-eigenvalue counts of every pivot, P_i, p_i, K_i, k_i and the
    pivots themselves (S_i = I + delta P_i, G_i) before factorization.
    """
    N, n, m = prob.N, prob.n, prob.m
    data = _data(prob)
    x = np.zeros((N + 1, n))
    u = np.zeros((N, m))
    y = np.zeros((N + 1, n))
    flags = np.zeros(N + 1, dtype=np.uint8)
    extra = {}
    if internals:
        extra = dict(neg_S=np.zeros(N + 1, np.int32), neg_G=np.zeros(N, np.int32),
                     P=np.zeros((N + 1, n, n)), p=np.zeros((N + 1, n)), K=np.zeros((N, m, n)),
                     k=np.zeros((N, m)), S=np.zeros((N + 1, n, n)), G=np.zeros((N, m, m)))
    e = lambda k, t=ctypes.c_double: _p(extra.get(k), t)  # noqa: E731
    st = _L().rlqr_orc_riccati(N, n, m, *[_p(a) for a in data], float(prob.delta), _p(x), _p(u),
                               _p(y), _p(flags, ctypes.c_uint8), e("neg_S", ctypes.c_int32),
                               e("neg_G", ctypes.c_int32), e("P"), e("p"), e("K"), e("k"),
                               e("S"), e("G"))
    return RiccatiResult(st, x, u, y, flags, **extra)


def riccati_batch(batch):
    """The same recursion on a uniform batch (leading axis = instance).

    ``batch`` has N, n, m, count, delta (count,) and stacked arrays.  Runs the
    instances in parallel with OpenMP; returns (status, x, u, y, flags)."""
    N, n, m, B = batch.N, batch.n, batch.m, batch.count
    data = _data(batch)
    delta = _f64(batch.delta)
    x = np.zeros((B, N + 1, n))
    u = np.zeros((B, N, m))
    y = np.zeros((B, N + 1, n))
    flags = np.zeros((B, N + 1), dtype=np.uint8)
    status = np.zeros(B, dtype=np.int32)
    _L().rlqr_orc_riccati_batch(B, N, n, m, *[_p(a) for a in data], _p(delta), _p(x), _p(u),
                                _p(y), _p(flags, ctypes.c_uint8), _p(status, ctypes.c_int32))
    return status, x, u, y, flags


# ----------------------------------------------------------------- dense KKT

def kkt_dims(N: int, n: int, m: int):
    """(number of primal unknowns N(n+m)+n, number of duals (N+1)n)."""
    return N * (n + m) + n, (N + 1) * n


def kkt_dense(prob):
    """Assemble K_LQR = [[P, C^T], [C, -Delta]] and b = [s; c] of eq.
    primal-dual-linear-system, with P, C, Delta, s, c laid out as in eq.
    optimal-control-specialization: primal order x_0, u_0, ..., x_{N-1},
    u_{N-1}, x_N, then duals y_0 .. y_N.  The system solved is K z = -b."""
    N, n, m = prob.N, prob.n, prob.m
    nxp, nyd = kkt_dims(N, n, m)
    dim = nxp + nyd
    K = np.zeros((dim, dim))
    b = np.zeros(dim)
    Q, M, R, q, r, A, B, c = _data(prob)

    def xo(i):
        return i * (n + m)

    def uo(i):
        return i * (n + m) + n

    def yo(i):
        return nxp + i * n

    for i in range(N + 1):
        K[xo(i):xo(i) + n, xo(i):xo(i) + n] = 0.5 * (Q[i] + Q[i].T)
        b[xo(i):xo(i) + n] = q[i]
        if i < N:
            K[xo(i):xo(i) + n, uo(i):uo(i) + m] = M[i]
            K[uo(i):uo(i) + m, xo(i):xo(i) + n] = M[i].T
            K[uo(i):uo(i) + m, uo(i):uo(i) + m] = 0.5 * (R[i] + R[i].T)
            b[uo(i):uo(i) + m] = r[i]
    # C: block row 0 is [-I 0 ...]; block row i+1 is [... A_i B_i -I ...]
    Cm = np.zeros((nyd, nxp))
    for i in range(N + 1):
        Cm[i * n:(i + 1) * n, xo(i):xo(i) + n] = -np.eye(n)
        if i < N:
            Cm[(i + 1) * n:(i + 2) * n, xo(i):xo(i) + n] = A[i]
            Cm[(i + 1) * n:(i + 2) * n, uo(i):uo(i) + m] = B[i]
        b[yo(i):yo(i) + n] = c[i]
    K[nxp:, :nxp] = Cm
    K[:nxp, nxp:] = Cm.T
    K[nxp:, nxp:] = -float(prob.delta) * np.eye(nyd)
    return K, b


class _Shallow:
    def __init__(self, prob, **kw):
        self.__dict__.update({k: getattr(prob, k) for k in
                              ("N", "n", "m", "Q", "M", "R", "q", "r", "A", "B", "c", "delta")})
        self.__dict__.update(kw)


def kkt_dense_diag(prob, dvec):
    """K and b of eq. primal-dual-linear-system with a general diagonal
    Delta_i = diag(dvec[i]) (dvec (N+1, n), positive) in place of delta I:
    the problem statement of Section "Dual-Regularized LQR" allows any
    symmetric positive-definite Delta_i."""
    K, b = kkt_dense(_Shallow(prob, delta=0.0))
    nxp, _ = kkt_dims(prob.N, prob.n, prob.m)
    K[nxp:, nxp:] = -np.diag(np.asarray(dvec, float).ravel())
    return K, b


def _ldl_d(S):
    """D of the unpivoted LDL^T of a symmetric matrix (the pivots)."""
    S = np.array(S, dtype=float)
    n = S.shape[0]
    d = np.zeros(n)
    L = np.eye(n)
    for j in range(n):
        d[j] = S[j, j] - np.sum(L[j, :j] ** 2 * d[:j])
        for i in range(j + 1, n):
            L[i, j] = (S[i, j] - np.sum(L[i, :j] * L[j, :j] * d[:j])) / d[j]
    return d


def riccati_diag(prob, dvec):
    """The sequential recursion of Theorem main-seq-theorem with a general
    diagonal Delta_i (numpy, plain): W = P (I + Delta P)^{-1}, g = p + W (c -
    Delta p), G = R + B^T W B, H = B^T W A + M^T, K = -G^{-1} H, k = -G^{-1} h,
    P = Q + A^T W A + H^T K, p = q + A^T g + H^T k; x_0 = (I + Delta_0 P_0)^{-1}
    (c_0 - Delta_0 p_0), u = K x + k, x_+ = (I + Delta P_+)^{-1}(A x + B u +
    c_+ - Delta p_+), y = P x + p.  Flags from the unpivoted LDL^T of
    S_i = I + Delta_i^{1/2} P_i Delta_i^{1/2} (Section "Inertia
    Certification") and of G_i.  Returns (x, u, y, flags)."""
    N, n, m = prob.N, prob.n, prob.m
    Q, M, R, q, r, A, B, c = _data(prob)
    D = [np.diag(np.asarray(dvec[i], float)) for i in range(N + 1)]
    Dh = [np.diag(np.sqrt(np.asarray(dvec[i], float))) for i in range(N + 1)]
    I = np.eye(n)
    P = [None] * (N + 1)
    p = [None] * (N + 1)
    K = [None] * N
    k = [None] * N
    flags = np.zeros(N + 1, dtype=np.uint8)
    P[N] = 0.5 * (Q[N] + Q[N].T)
    p[N] = q[N].copy()
    for i in range(N - 1, -1, -1):
        Pn = P[i + 1]
        Wm = Pn @ np.linalg.inv(I + D[i + 1] @ Pn)
        Wm = 0.5 * (Wm + Wm.T)
        g = p[i + 1] + Wm @ (c[i + 1] - D[i + 1] @ p[i + 1])
        G = 0.5 * (R[i] + R[i].T) + B[i].T @ Wm @ B[i]
        H = B[i].T @ Wm @ A[i] + M[i].T
        h = r[i] + B[i].T @ g
        if np.all(_ldl_d(G) > 0):
            flags[i] |= 2
        K[i] = -np.linalg.solve(G, H)
        k[i] = -np.linalg.solve(G, h)
        Pi = 0.5 * (Q[i] + Q[i].T) + A[i].T @ Wm @ A[i] + H.T @ K[i]
        P[i] = 0.5 * (Pi + Pi.T)
        p[i] = q[i] + A[i].T @ g + H.T @ k[i]
    flags[N] |= 2
    for i in range(N + 1):
        if np.all(_ldl_d(I + Dh[i] @ P[i] @ Dh[i]) > 0):
            flags[i] |= 1
    x = np.zeros((N + 1, n))
    u = np.zeros((N, m))
    x[0] = np.linalg.solve(I + D[0] @ P[0], c[0] - D[0] @ p[0])
    for i in range(N):
        u[i] = K[i] @ x[i] + k[i]
        x[i + 1] = np.linalg.solve(I + D[i + 1] @ P[i + 1],
                                   A[i] @ x[i] + B[i] @ u[i] + c[i + 1] - D[i + 1] @ p[i + 1])
    y = np.stack([P[i] @ x[i] + p[i] for i in range(N + 1)])
    return x, u, y, flags


def split_solution(prob, z):
    """Split z (primal then dual, as in kkt_dense) into x, u, y arrays."""
    N, n, m = prob.N, prob.n, prob.m
    nxp, _ = kkt_dims(N, n, m)
    x = np.zeros((N + 1, n))
    u = np.zeros((N, m))
    for i in range(N + 1):
        x[i] = z[i * (n + m):i * (n + m) + n]
        if i < N:
            u[i] = z[i * (n + m) + n:(i + 1) * (n + m)]
    y = z[nxp:].reshape(N + 1, n).copy()
    return x, u, y


def join_solution(prob, x, u, y):
    """Inverse of split_solution."""
    N, n, m = prob.N, prob.n, prob.m
    parts = []
    for i in range(N + 1):
        parts.append(np.asarray(x[i], dtype=np.float64))
        if i < N:
            parts.append(np.asarray(u[i], dtype=np.float64))
    parts.append(np.asarray(y, dtype=np.float64).reshape(-1))
    return np.concatenate(parts)


def cross_stage_solve(prob, Jq, Jr, Jc, H, r_theta):
    """Section "Cross-Stage Variables", eq. cross-stage-kkt: with K, b of
    ``kkt_dense`` and the p columns of J_theta given in the layout of the
    right-hand side (Jq: (p, N+1, n) pairs with x, Jr: (p, N, m) with u,
    Jc: (p, N+1, n) with y), solve [[K, J], [J^T, H]] [dw; dtheta] =
    -[b; r_theta] densely.  Returns (x, u, y) of dw and dtheta."""
    K, b = kkt_dense(prob)
    p = len(r_theta)
    J = np.stack([join_solution(prob, Jq[j], Jr[j], Jc[j]) for j in range(p)], axis=1)
    dim = K.shape[0]
    big = np.zeros((dim + p, dim + p))
    big[:dim, :dim] = K
    big[:dim, dim:] = J
    big[dim:, :dim] = J.T
    big[dim:, dim:] = np.asarray(H, dtype=np.float64)
    rhs = -np.concatenate([b, np.asarray(r_theta, dtype=np.float64)])
    sol = np.linalg.solve(big, rhs)
    x, u, y = split_solution(prob, sol[:dim])
    return x, u, y, sol[dim:]


def bk_factor(K):
    """Bunch-Kaufman P K P^T = L D L^T (copy of K factored in place)."""
    F = _f64(K).copy()
    dim = F.shape[0]
    perm = np.zeros(dim, np.int32)
    bsize = np.zeros(dim, np.int32)
    zero = _L().rlqr_orc_bk_factor(dim, _p(F), _p(perm, ctypes.c_int32),
                                   _p(bsize, ctypes.c_int32))
    return F, perm, bsize, zero


def bk_solve(fac, rhs):
    F, perm, bsize, _ = fac
    x = _f64(rhs).copy()
    _L().rlqr_orc_bk_solve(F.shape[0], _p(F), _p(perm, ctypes.c_int32),
                           _p(bsize, ctypes.c_int32), _p(x))
    return x


def bk_inertia(fac):
    F, _, bsize, _ = fac
    inertia = np.zeros(3, np.int32)
    _L().rlqr_orc_bk_inertia(F.shape[0], _p(F), _p(bsize, ctypes.c_int32),
                             _p(inertia, ctypes.c_int32))
    return tuple(int(v) for v in inertia)


def dense_solve(prob, refine: int = 1):
    """Unique solution of K z = -b (eq. primal-dual-linear-system) by
    Bunch-Kaufman, plus ``refine`` steps of FP64 iterative refinement, and the
    inertia (n_plus, n_minus, n_zero) from D.  Returns (x, u, y, inertia)."""
    K, b = kkt_dense(prob)
    fac = bk_factor(K)
    z = bk_solve(fac, -b)
    for _ in range(refine):
        z = z - bk_solve(fac, K @ z + b)
    x, u, y = split_solution(prob, z)
    return x, u, y, bk_inertia(fac)


def jacobi_inertia(Kmat, tau=None, max_sweeps: int = 60):
    """(n_plus, n_minus, n_zero) of a symmetric matrix from cyclic Jacobi
    eigenvalues, counting |lambda| <= tau as zero (default tau = 1e3 eps
    ||K||_F).  Also returns the eigenvalues."""
    A = _f64(Kmat).copy()
    dim = A.shape[0]
    if tau is None:
        tau = 1e3 * np.finfo(float).eps * float(np.sqrt((A * A).sum()))
    inertia = np.zeros(3, np.int32)
    eig = np.zeros(dim)
    _L().rlqr_orc_jacobi_inertia(dim, _p(A), float(tau), max_sweeps,
                                 _p(inertia, ctypes.c_int32), _p(eig))
    return tuple(int(v) for v in inertia), eig


def band_solve(prob):
    """Solve eq. primal-dual-linear-system by banded LU with partial pivoting
    in the order (y_0, x_0, u_0, ..., y_N, x_N).  Returns (status, x, u, y)."""
    N, n, m = prob.N, prob.n, prob.m
    x = np.zeros((N + 1, n))
    u = np.zeros((N, m))
    y = np.zeros((N + 1, n))
    st = _L().rlqr_orc_band_solve(N, n, m, *[_p(a) for a in _data(prob)], float(prob.delta),
                                  _p(x), _p(u), _p(y))
    return st, x, u, y


@dataclass
class Residual:
    res_q: np.ndarray
    res_r: np.ndarray
    res_c: np.ndarray
    rmax: float
    kmax: float
    zmax: float
    bmax: float
    rel: float


def residual(prob, x, u, y) -> Residual:
    """Residual K z + b of Section "Residual Computation" for the given
    (x, u, y), and the normwise backward error
    rel = ||K z + b||_inf / (||K||_inf ||z||_inf + ||b||_inf)."""
    N, n, m = prob.N, prob.n, prob.m
    rq = np.zeros((N + 1, n))
    rr = np.zeros((N, m))
    rc = np.zeros((N + 1, n))
    norms = np.zeros(5)
    _L().rlqr_orc_residual(N, n, m, *[_p(a) for a in _data(prob)], float(prob.delta),
                           _p(_f64(x)), _p(_f64(u)), _p(_f64(y)), _p(rq), _p(rr), _p(rc),
                           _p(norms))
    return Residual(rq, rr, rc, *[float(v) for v in norms])


def forward_error(ref, x, u, y):
    """||z - z_ref||_inf / ||z_ref||_inf over (x, u, y)."""
    rx, ru, ry = ref
    num = max(np.abs(np.asarray(x) - rx).max(), np.abs(np.asarray(u) - ru).max(),
              np.abs(np.asarray(y) - ry).max())
    den = max(np.abs(rx).max(), np.abs(ru).max(), np.abs(ry).max())
    return float(num / den) if den > 0 else float(num)
