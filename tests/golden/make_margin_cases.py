"""Write margin_cases.json: instances whose certificate has one pivot placed
at a chosen relative margin, decided by the FP64 oracle only.

Each case takes the seeded generic instance inputs.random_instance(seed, N,
n, m, delta) and moves ONE pivot matrix X of stage k* so that its eigenvalue
closest to zero sits at  sign * mu * ||X||_2  (sign +1: positive definite
with margin mu; sign -1: one negative eigenvalue of relative size mu):
  * kind "G" (control pivot G_{k*} = R_{k*} + B^T W_{k*+1} B):
        R_{k*} <- R_{k*} - alpha I, which shifts G_{k*} by -alpha I and leaves
        every later stage unchanged (W_{k*+1} does not depend on R_{k*});
  * kind "S" (state pivot I + delta P_0 of the initial stage, k* = 0):
        Q_0 <- Q_0 - alpha I, which shifts P_0 by -alpha I and I + delta P_0
        by -delta alpha I, and changes no other pivot.
With lambda_1 <= ... <= lambda_n the eigenvalues of X before the shift and
s = sign, alpha solves (lambda_1 - a) / (lambda_n - a) = s mu:
        a = (lambda_1 - s mu lambda_n) / (1 - s mu)     (alpha = a / delta for "S").
Every other pivot of the case must keep min |lambda| >= 1e-3 ||X||_2 (else
the next seed is tried), so that the chosen pivot is the only one near its
decision boundary.  The tests compare the GPU's flags with the oracle's,
byte for byte, at every margin.  Each case also records scaled_margin, the
smallest eigenvalue of the oracle's pivot in Jacobi scaling (D^-1/2 X D^-1/2,
D = diag(max(|X_jj|, 2^-24 max_j |X_jj|))): the quantity that the mixed
path's certificate margin is stated in.

Usage: python tests/golden/make_margin_cases.py   (rewrites the JSON next to it)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2509_16370_b300 import inputs  # noqa: E402

OTHER_MARGIN = 1e-3
MUS = (1e-3, 1e-5, 1e-7)
SHAPES = [  # (N, n, m, delta, k* of the G cases)
    (64, 12, 4, 1e-3, 40),
    (48, 6, 2, 1e-2, 17),
]


def margins(res):
    es = np.linalg.eigvalsh(res.S)
    eg = np.linalg.eigvalsh(res.G)
    return (np.abs(es).min(-1) / np.abs(es).max(-1), np.abs(eg).min(-1) / np.abs(eg).max(-1),
            es, eg)


def jacobi_lambda_min(X):
    dg = np.abs(np.diag(X))
    d = np.maximum(dg, 2.0 ** -24 * dg.max())
    s = 1.0 / np.sqrt(d)
    return float(np.linalg.eigvalsh(s[:, None] * X * s[None, :]).min())


def shifted(p, kind, kstar, alpha):
    q = inputs.Problem(p.N, p.n, p.m, p.Q.copy(), p.M, p.R.copy(), p.q, p.r, p.A, p.B, p.c,
                       p.delta)
    if kind == "G":
        q.R[kstar] -= alpha * np.eye(p.m)
    else:
        q.Q[kstar] -= alpha * np.eye(p.n)
    return q


def make_case(kind, sign, mu, N, n, m, delta, kg, seed0):
    for seed in range(seed0, seed0 + 400):
        p = inputs.random_instance(seed, N, n, m, delta)
        res = oracle.riccati(p, internals=True)
        if res.status != oracle.OK:
            continue
        ms, mg, _, _ = margins(res)
        if ms.min() < OTHER_MARGIN or mg.min() < OTHER_MARGIN:
            continue
        kstar = kg if kind == "G" else 0
        X = res.G[kstar] if kind == "G" else res.S[kstar]
        lam = np.linalg.eigvalsh(X)
        a = (lam[0] - sign * mu * lam[-1]) / (1.0 - sign * mu)
        alpha = float(a if kind == "G" else a / delta)
        q = shifted(p, kind, kstar, alpha)
        r2 = oracle.riccati(q, internals=True)
        if r2.status not in (oracle.OK, oracle.NOT_PD):
            continue
        ms2, mg2, es2, eg2 = margins(r2)
        # the chosen pivot at its margin (to rounding), every other pivot clear
        ev = eg2[kstar] if kind == "G" else es2[kstar]
        got = ev[np.argmin(np.abs(ev))] / np.abs(ev).max()
        if abs(got - sign * mu) > 1e-3 * mu:
            continue
        other_s = np.delete(ms2, kstar) if kind == "S" else ms2
        other_g = np.delete(mg2, kstar) if kind == "G" else mg2
        if other_s.min() < OTHER_MARGIN or other_g.min() < OTHER_MARGIN:
            continue
        return dict(kind=kind, sign=sign, mu=mu, seed=seed, N=N, n=n, m=m, delta=delta,
                    kstar=kstar, alpha=alpha, margin=float(got),
                    scaled_margin=jacobi_lambda_min(r2.G[kstar] if kind == "G" else r2.S[kstar]),
                    oracle_flags_at_kstar=int(r2.flags[kstar]))
    raise RuntimeError(f"no instance for {kind} {sign} {mu} {(N, n, m)}")


def main():
    cases = []
    for si, (N, n, m, delta, kg) in enumerate(SHAPES):
        for kind in ("G", "S"):
            for sign in (1, -1):
                for mu in MUS:
                    cases.append(make_case(kind, sign, mu, N, n, m, delta, kg, 1000 * (si + 1)))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "margin_cases.json")
    with open(out, "w") as f:
        json.dump({"rule": __doc__.split("\n\n")[1], "cases": cases}, f, indent=1)
    print(f"{len(cases)} cases -> {out}")


if __name__ == "__main__":
    main()
