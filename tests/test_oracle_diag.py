"""Pins of the oracle's general diagonal dual regularization (CPU): the
recursion against the dense solve of eq. primal-dual-linear-system with
Delta_i = diag(d_i) (the plain definition), the scalar case against the C
recursion, and the flags against the eigenvalue inertia of the dense matrix
(Theorem riccati-inertia-certification-theorem: all pivots PD iff the
inertia is (N(n+m)+n, (N+1)n, 0))."""
import numpy as np
import pytest

import oracle
from paper_2509_16370_b300 import inputs


def _case(seed, N, n, m, lo=-5.0, hi=-1.0):
    prob = inputs.random_instance(seed, N, n, m, 1e-3)
    d = 10.0 ** np.random.default_rng(seed).uniform(lo, hi, (N + 1, n))
    return prob, d


@pytest.mark.parametrize("shape", [(10, 4, 2), (7, 6, 3), (16, 3, 1)])
def test_recursion_matches_the_dense_solve(shape):
    prob, d = _case(41, *shape)
    x, u, y, flags = oracle.riccati_diag(prob, d)
    K, b = oracle.kkt_dense_diag(prob, d)
    z = np.linalg.solve(K, -b)
    xr, ur, yr = oracle.split_solution(prob, z)
    scale = max(1.0, np.abs(z).max())
    for a, r in ((x, xr), (u, ur), (y, yr)):
        assert np.abs(a - r).max() <= 1e-10 * scale


def test_scalar_case_is_the_plain_recursion():
    prob = inputs.random_instance(42, 12, 4, 2, 3e-3)
    d = np.full((13, 4), prob.delta)
    x, u, y, flags = oracle.riccati_diag(prob, d)
    ref = oracle.riccati(prob)
    np.testing.assert_array_equal(flags, ref.flags)
    assert np.abs(x - ref.x).max() <= 1e-12 * max(1, np.abs(ref.x).max())


def test_flags_match_the_eigenvalue_inertia():
    seen = set()
    for seed in range(12):
        prob, d = _case(100 + seed, 8, 4, 2, -3.0, 1.0)
        if seed % 2:
            Q = prob.Q.copy()
            Q -= 3.0 * np.eye(4)           # indefinite costs: some pivots fail
            prob.Q = Q
        x, u, y, flags = oracle.riccati_diag(prob, d)
        K, _ = oracle.kkt_dense_diag(prob, d)
        ev = np.linalg.eigvalsh(K)
        N, n, m = prob.N, prob.n, prob.m
        ok = bool(np.all(flags == 3))
        correct = (int((ev > 0).sum()), int((ev < 0).sum())) == (N * (n + m) + n, (N + 1) * n)
        assert ok == correct
        seen.add(ok)
    assert seen == {True, False}
