"""FP64 restatement of the paper's parallel formulation (Section "Parallel
Algorithm"), for the parity tests of the associative-scan path.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use it; it shares
nothing with the CUDA library.  Plain numpy in FP64; ``numpy.linalg.solve``
is the only library step.  Everything follows the paper's notation:

* ``stage_element(prob, i)`` -- the interval element (P, p, A, C, c)_{i->i+1}
  of eq. lqr-gpu-init-running (i < N) and eq. lqr-gpu-init-terminal (i = N),
  after the control variables are eliminated (Section "Parallel Algorithm").
* ``combine(e_ij, e_jk)`` -- the combination rule of eq. lqr-gpu-combo for an
  earlier interval (i -> j) and a later one (j -> k).
* ``value_functions(prob)`` -- P_i = P_{i->N+1} and p_i = p_{i->N+1} for all
  i, as the reverse fold S_i = e_i (+) S_{i+1} with S_N = e_N (what the
  reverse associative scan computes; the fold order is the plain definition).
* ``chunk_boundaries(prob, L)`` -- the same P_i, p_i at the starts of
  chunks of L stages, by composing each chunk's elements first and folding
  the chunk elements afterwards (the order of a chunked scan; it exercises
  the combination rule with general later intervals, A_jk, C_jk != 0).
* ``p_recurrence(...)`` -- Corollary p-recurrence.
* ``compose_affine(maps)`` -- the forward composition of Section "Composing
  Affine Functions with Associative Scans": f((a, B), (c, D)) = (Da + c, DB).
* ``solution(prob)`` -- x, u, y from the value functions: W, K, k (Theorem
  main-seq-theorem, eq. value-fn-formulas, control-law), x_0 (eq.
  recover-x0), the affine maps x_{i+1} = E_i x_i + e_i composed with
  ``compose_affine`` and applied to x_0, u_i = K_i x_i + k_i and
  y_i = P_i x_i + p_i.

The scan path additionally needs every R_i invertible (the elimination of
u_i divides by R_i).
"""
from __future__ import annotations

import numpy as np


def stage_element(prob, i):
    """(P, p, A, C, c)_{i -> i+1}; eq. lqr-gpu-init-running / -terminal."""
    n = prob.n
    if i == prob.N:
        Z = np.zeros((n, n))
        return (np.array(prob.Q[i], dtype=float), np.array(prob.q[i], dtype=float), Z, Z.copy(),
                np.zeros(n))
    Q, M, R = prob.Q[i], prob.M[i], prob.R[i]
    A, B = prob.A[i], prob.B[i]
    q, r, c_next = prob.q[i], prob.r[i], prob.c[i + 1]
    Rinv_MT = np.linalg.solve(R, M.T)   # R^{-1} M^T
    Rinv_BT = np.linalg.solve(R, B.T)   # R^{-1} B^T
    Rinv_r = np.linalg.solve(R, r)      # R^{-1} r
    P = Q - M @ Rinv_MT
    p = q - M @ Rinv_r
    Ai = A - B @ Rinv_MT
    C = prob.delta * np.eye(n) + B @ Rinv_BT
    c = c_next - B @ Rinv_r
    return P, p, Ai, C, c


def combine(e_ij, e_jk):
    """Eq. lqr-gpu-combo: the element of interval i -> k from i -> j and j -> k."""
    P1, p1, A1, C1, c1 = e_ij
    P2, p2, A2, C2, c2 = e_jk
    n = P1.shape[0]
    I = np.eye(n)
    IPC = I + P2 @ C1          # I + P_jk C_ij
    ICP = I + C1 @ P2          # I + C_ij P_jk
    P = A1.T @ np.linalg.solve(IPC, P2) @ A1 + P1
    p = A1.T @ np.linalg.solve(IPC, p2 + P2 @ c1) + p1
    A = A2 @ np.linalg.solve(ICP, A1)
    C = A2 @ np.linalg.solve(ICP, C1) @ A2.T + C2
    c = A2 @ np.linalg.solve(ICP, c1 - C1 @ p2) + c2
    return P, p, A, C, c


def value_functions(prob):
    """P_i, p_i (i = 0..N) from the reverse fold of the interval elements."""
    N = prob.N
    S = stage_element(prob, N)
    P = [None] * (N + 1)
    p = [None] * (N + 1)
    P[N], p[N] = S[0], S[1]
    for i in range(N - 1, -1, -1):
        S = combine(stage_element(prob, i), S)
        P[i], p[i] = S[0], S[1]
    return np.array(P), np.array(p)


def chunk_boundaries(prob, L):
    """(starts, P, p): P_s, p_s at every chunk start s = 0, L, 2L, ... < N.

    Chunk c holds the elements of stages [cL, min(cL + L, N)); its element is
    their left-to-right composition; the terminal element e_N is the last
    item of the fold over chunks."""
    N = prob.N
    starts = list(range(0, N, L))
    chunk = []
    for s0 in starts:
        e = stage_element(prob, s0)
        for i in range(s0 + 1, min(s0 + L, N)):
            e = combine(e, stage_element(prob, i))
        chunk.append(e)
    S = stage_element(prob, N)
    P = [None] * len(starts)
    p = [None] * len(starts)
    for c in range(len(starts) - 1, -1, -1):
        S = combine(chunk[c], S)
        P[c], p[c] = S[0], S[1]
    return np.array(starts), np.array(P), np.array(p)


def factor_from_P(prob, P):
    """W_{i+1}, G_i, K_i from the value functions (Theorem main-seq-theorem,
    eq. value-fn-formulas): W = (I + delta P)^{-1} P, G = R + B^T W B,
    H = B^T W A + M^T, K = -G^{-1} H.  Returns W (N+1 entries), K."""
    N, n = prob.N, prob.n
    I = np.eye(n)
    W = np.array([np.linalg.solve(I + prob.delta * P[i], P[i]) for i in range(N + 1)])
    K = []
    for i in range(N):
        Wn = W[i + 1]
        G = prob.R[i] + prob.B[i].T @ Wn @ prob.B[i]
        H = prob.B[i].T @ Wn @ prob.A[i] + prob.M[i].T
        K.append(-np.linalg.solve(G, H))
    return W, np.array(K)


def p_recurrence(prob, W, K, q=None, r=None, c=None):
    """Corollary p-recurrence for a right-hand side (q, r, c) (defaults: the
    problem's): p_N = q_N, p_k = q_k + K_k^T r_k + (A_k + B_k K_k)^T
    (p_{k+1} + W_{k+1} (c_{k+1} - delta p_{k+1}))."""
    q = prob.q if q is None else q
    r = prob.r if r is None else r
    c = prob.c if c is None else c
    N = prob.N
    p = [None] * (N + 1)
    p[N] = np.array(q[N], dtype=float)
    for k in range(N - 1, -1, -1):
        g = p[k + 1] + W[k + 1] @ (c[k + 1] - prob.delta * p[k + 1])
        ABK = prob.A[k] + prob.B[k] @ K[k]
        p[k] = q[k] + K[k].T @ r[k] + ABK.T @ g
    return np.array(p)


def compose_affine(maps):
    """Forward composition of affine maps F_i(x) = M_i x + m_i given as
    (m_i, M_i): returns [F_0, F_1 o F_0, ...] as (offset, matrix) pairs, with
    f((a, B), (c, D)) = (D a + c, D B)."""
    out = []
    acc = None
    for m_i, M_i in maps:
        acc = (m_i, M_i) if acc is None else (M_i @ acc[0] + m_i, M_i @ acc[1])
        out.append(acc)
    return out


def solution(prob):
    """x, u, y and the value functions by the parallel formulation's steps."""
    N, n = prob.N, prob.n
    I = np.eye(n)
    P, p_scan = value_functions(prob)
    W, K = factor_from_P(prob, P)
    p = p_recurrence(prob, W, K)
    k = []
    for i in range(N):
        G = prob.R[i] + prob.B[i].T @ W[i + 1] @ prob.B[i]
        g = p[i + 1] + W[i + 1] @ (prob.c[i + 1] - prob.delta * p[i + 1])
        h = prob.r[i] + prob.B[i].T @ g
        k.append(-np.linalg.solve(G, h))
    k = np.array(k)
    # eq. recover-x0: x_0 = (I + delta P_0)^{-1} (c_0 - delta p_0)
    x0 = np.linalg.solve(I + prob.delta * P[0], prob.c[0] - prob.delta * p[0])
    maps = []
    for i in range(N):
        S_inv_ABK = np.linalg.solve(I + prob.delta * P[i + 1], prob.A[i] + prob.B[i] @ K[i])
        e_i = np.linalg.solve(I + prob.delta * P[i + 1],
                              prob.B[i] @ k[i] + prob.c[i + 1] - prob.delta * p[i + 1])
        maps.append((e_i, S_inv_ABK))
    comp = compose_affine(maps)
    x = np.zeros((N + 1, n))
    x[0] = x0
    for i in range(N):
        x[i + 1] = comp[i][1] @ x0 + comp[i][0]
    u = np.array([K[i] @ x[i] + k[i] for i in range(N)])
    y = np.array([P[i] @ x[i] + p[i] for i in range(N + 1)])
    return dict(x=x, u=u, y=y, P=P, p=p, p_scan=p_scan, W=W, K=K, k=k)
