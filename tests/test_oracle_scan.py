"""Pins of the oracle's restatement of the parallel formulation
(``oracle/scan.py``, Section "Parallel Algorithm") to things other than itself:

* the value functions from the fold of eq. lqr-gpu-combo, and from a
  chunked fold (elements composed within chunks first, which exercises the
  rule with general later intervals), equal the sequential recursion's P_i
  and p_i (eq. value-fn-formulas), which the paper states and which is
  pinned in test_oracle_pins.py;
* x, u, y from the parallel steps equal numpy's solve of the assembled KKT
  system (the plain definition);
* the combination rule and the affine composition are associative (the
  property the scans rely on), checked on random elements;
* planted mistakes in the combination rule (a transposed A, a dropped C, a
  sign flip in c) break the first pin.
"""
import numpy as np
import pytest

import oracle
from oracle import scan
from paper_2509_16370_b300 import inputs


def _instances():
    out = [inputs.random_instance(201, 12, 4, 2, 0.3, with_M=True),
           inputs.random_instance(202, 20, 3, 3, 1e-3, with_M=False),
           inputs.random_instance(203, 9, 5, 2, 2.0, with_M=True)]
    p = inputs.random_instance(204, 15, 4, 2, 0.05, with_M=True)
    p.Q[3] -= 1.5 * np.eye(4)  # a non-convex stage
    out.append(p)
    return out


@pytest.mark.parametrize("idx", range(4))
def test_value_functions_equal_sequential_recursion(idx):
    p = _instances()[idx]
    r = oracle.riccati(p, internals=True)
    P, p_scan = scan.value_functions(p)
    scale = max(1.0, np.abs(r.P).max())
    np.testing.assert_allclose(P, r.P, atol=1e-10 * scale)
    np.testing.assert_allclose(p_scan, r.p, atol=1e-10 * max(1.0, np.abs(r.p).max()))


@pytest.mark.parametrize("idx,L", [(0, 4), (1, 3), (2, 2), (3, 5), (1, 7)])
def test_chunked_fold_equals_sequential_recursion(idx, L):
    p = _instances()[idx]
    r = oracle.riccati(p, internals=True)
    starts, P, p_c = scan.chunk_boundaries(p, L)
    np.testing.assert_allclose(P, r.P[starts], atol=1e-10 * max(1.0, np.abs(r.P).max()))
    np.testing.assert_allclose(p_c, r.p[starts], atol=1e-10 * max(1.0, np.abs(r.p).max()))


@pytest.mark.parametrize("idx", range(4))
def test_parallel_solution_equals_kkt_solve(idx):
    p = _instances()[idx]
    K, b = oracle.kkt_dense(p)
    x, u, y = oracle.split_solution(p, np.linalg.solve(K, -b))
    sol = scan.solution(p)
    fe = oracle.forward_error((x, u, y), sol["x"], sol["u"], sol["y"])
    assert fe < 1e-9
    # the p-recurrence reproduces the p of the combination rule
    np.testing.assert_allclose(sol["p"], sol["p_scan"],
                               atol=1e-10 * max(1.0, np.abs(sol["p"]).max()))


def _random_element(rng, n):
    G = rng.standard_normal((n, n))
    P = G @ G.T + 0.1 * np.eye(n)
    H = rng.standard_normal((n, n))
    C = H @ H.T * 0.2 + 0.05 * np.eye(n)
    return (P, rng.standard_normal(n), rng.standard_normal((n, n)) * 0.6, C, rng.standard_normal(n))


def test_combine_is_associative():
    rng = np.random.default_rng(5)
    for _ in range(5):
        e1, e2, e3 = (_random_element(rng, 4) for _ in range(3))
        left = scan.combine(scan.combine(e1, e2), e3)
        right = scan.combine(e1, scan.combine(e2, e3))
        for a, b in zip(left, right):
            np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-10)


def test_affine_composition():
    """compose_affine gives F_i o ... o F_0 (checked against applying the maps
    one after another) and its operator is associative."""
    rng = np.random.default_rng(6)
    maps = [(rng.standard_normal(3), rng.standard_normal((3, 3))) for _ in range(6)]
    comp = scan.compose_affine(maps)
    x0 = rng.standard_normal(3)
    x = x0.copy()
    for i, (m_i, M_i) in enumerate(maps):
        x = M_i @ x + m_i
        np.testing.assert_allclose(comp[i][1] @ x0 + comp[i][0], x, rtol=1e-12, atol=1e-12)

    def f(a, b):
        return (b[1] @ a[0] + b[0], b[1] @ a[1])
    a, b, c = maps[:3]
    l, r = f(f(a, b), c), f(a, f(b, c))
    np.testing.assert_allclose(l[0], r[0], atol=1e-12)
    np.testing.assert_allclose(l[1], r[1], atol=1e-12)


@pytest.mark.parametrize("mutation", ["transpose_A1", "drop_C2", "flip_c"])
def test_pins_detect_mistakes_in_the_combination_rule(mutation, monkeypatch):
    p = _instances()[0]
    r = oracle.riccati(p, internals=True)
    good = scan.combine

    def bad(e_ij, e_jk):
        P1, p1, A1, C1, c1 = e_ij
        P2, p2, A2, C2, c2 = e_jk
        if mutation == "transpose_A1":
            A1 = A1.T
        elif mutation == "drop_C2":
            C2 = np.zeros_like(C2)
        elif mutation == "flip_c":
            c1 = -c1
        return good((P1, p1, A1, C1, c1), (P2, p2, A2, C2, c2))
    monkeypatch.setattr(scan, "combine", bad)
    starts, P, p_c = scan.chunk_boundaries(p, 4)
    err = max(np.abs(P - r.P[starts]).max() / np.abs(r.P).max(),
              np.abs(p_c - r.p[starts]).max() / np.abs(r.p).max())
    assert err > 1e-3
