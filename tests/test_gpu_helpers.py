"""GPU tests of the device helpers behind the mixed-precision path, each
against an independent definition computed on the host:

* f64_to_f32_rz: numpy's round-to-nearest FP32 value stepped toward zero
  when it overshoots (round toward zero), with the stated flush rules;
* f32_to_f64: numpy's exact widening (FP32 subnormals flush to zero);
* split_f64: hi equals the truncation and hi + lo is within 2^-46 |v|;
* the float-float dot product: within the bound derived from its error
  terms of the exact rational dot product (fractions.Fraction);
* recip_pivot: within one FP32 ulp of the exact reciprocal;
* gershgorin_row_pd: sound (a pass implies the exact rational test
  1 + delta (P_ii - sum |P_ij|) > 0) and not needlessly conservative.
* warp_pd_proof_f32: sound (a pass implies that the smallest eigenvalue of
  I + delta P - tau D, D its diagonal, computed by LAPACK in FP64 from the
  exact FP32 P, is positive), invariant to diagonal scaling, and passing
  every matrix whose Jacobi-scaled smallest eigenvalue is clear of tau.
"""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = tmp_path_factory.mktemp("probe") / "helpers_probe.so"
    cmd = ["nvcc", "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
           "-Xcompiler", "-fPIC", "-shared", "-o", str(out),
           os.path.join(HERE, "csrc", "helpers_probe.cu")]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(str(out))
    for name in ("probe_conv", "probe_widen", "probe_ffdot", "probe_recip", "probe_gersh",
                 "probe_pdproof"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _test_doubles(rng):
    mag = np.exp2(rng.uniform(-140.0, 140.0, 20000)) * rng.uniform(1.0, 2.0, 20000)
    v = mag * rng.choice([-1.0, 1.0], mag.size)
    f32max = float(np.finfo(np.float32).max)
    special = [0.0, -0.0, np.inf, -np.inf, np.nan, 2.0 ** -126, -(2.0 ** -126),
               np.nextafter(2.0 ** -126, 0.0), 2.0 ** 128, np.nextafter(2.0 ** 128, 0.0),
               f32max, -f32max, 1.0, -1.0, 1.0 + 2.0 ** -30, 1.0 - 2.0 ** -40,
               2.0 ** -80, np.nextafter(2.0 ** -80, 0.0), 3.0, 0.1, -0.1]
    return np.concatenate([v, np.array(special)])


def _rz_expected(v):
    with np.errstate(over="ignore", invalid="ignore"):
        f = v.astype(np.float32)
        over = np.abs(f.astype(np.float64)) > np.abs(v)
        f[over] = np.nextafter(f[over], np.float32(0.0))
    a = np.abs(v)
    f[a < 2.0 ** -126] = np.copysign(np.float32(0.0), v[a < 2.0 ** -126])
    f[(a >= 2.0 ** 128) & ~np.isnan(v)] = np.copysign(np.float32(np.inf), v[(a >= 2.0 ** 128) & ~np.isnan(v)])
    return f


def test_integer_conversions_and_split(probe):
    rng = np.random.default_rng(7)
    v = _test_doubles(rng)
    dv = _dev(v)
    rz = torch.empty(v.size, dtype=torch.float32, device="cuda")
    hi = torch.empty_like(rz)
    lo = torch.empty_like(rz)
    assert probe.probe_conv(_ptr(dv), _ptr(rz), _ptr(hi), _ptr(lo), v.size) == 0
    rz, hi, lo = rz.cpu().numpy(), hi.cpu().numpy(), lo.cpu().numpy()
    exp = _rz_expected(v)
    nan = np.isnan(v)
    assert np.all(np.isnan(rz[nan]))
    np.testing.assert_array_equal(rz[~nan].view(np.uint32), exp[~nan].view(np.uint32))
    np.testing.assert_array_equal(hi[~nan].view(np.uint32), exp[~nan].view(np.uint32))
    # hi + lo is exact in FP64 (at most 47 significant bits) and so is v - (hi + lo)
    fin = np.isfinite(v) & (np.abs(v) < 2.0 ** 128)
    err = np.abs(v[fin] - (hi[fin].astype(np.float64) + lo[fin].astype(np.float64)))
    a = np.abs(v[fin])
    bound = np.where(a >= 2.0 ** -80, a * 2.0 ** -46, 2.0 ** -103)
    assert np.all(err <= bound)


def test_f32_to_f64_widening(probe):
    rng = np.random.default_rng(8)
    bits = rng.integers(0, 2 ** 32, 50000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    extra = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-40, 1.17549435e-38, 3.4e38],
                     dtype=np.float32)
    f = np.concatenate([f, extra])
    df = _dev(f)
    w = torch.empty(f.size, dtype=torch.float64, device="cuda")
    assert probe.probe_widen(_ptr(df), _ptr(w), f.size) == 0
    w = w.cpu().numpy()
    with np.errstate(invalid="ignore"):
        exp = f.astype(np.float64)
    sub = (np.abs(f) < np.finfo(np.float32).tiny) & (f != 0)
    exp[sub] = np.copysign(0.0, exp[sub])
    nan = np.isnan(f)
    assert np.all(np.isnan(w[nan]))
    np.testing.assert_array_equal(w[~nan].view(np.uint64), exp[~nan].view(np.uint64))


def test_float_float_dot_product(probe):
    rng = np.random.default_rng(9)
    rows, length = 96, 28
    a = rng.standard_normal((rows, length)) * np.exp2(rng.uniform(-20, 20, (rows, length)))
    z = rng.standard_normal(length) * np.exp2(rng.uniform(-10, 10, length))
    b = rng.standard_normal(rows) * 1e3
    a[:8] *= 1e-30  # tiny entries
    out = torch.empty(rows, dtype=torch.float64, device="cuda")
    assert probe.probe_ffdot(_ptr(_dev(a)), _ptr(_dev(z)), _ptr(_dev(b)), rows, length, _ptr(out)) == 0
    out = out.cpu().numpy()
    errs = []
    for r in range(rows):
        exact = Fraction(b[r]) + sum(Fraction(a[r, j]) * Fraction(z[j]) for j in range(length))
        scale = abs(b[r]) + float(np.sum(np.abs(a[r] * z)))
        # split errors 3 * 2^-46 per term, two-sum exact, the low-part sum
        # (len^2 + 4 len) * 2^-48 of the sum of magnitudes in the worst case
        bound = (3 * 2.0 ** -46 + (length ** 2 + 4 * length) * 2.0 ** -48) * scale + 2.0 ** -100
        e = abs(Fraction(out[r]) - exact)
        assert e <= Fraction(bound), (r, float(e), bound)
        errs.append(float(e) / scale)
    # typical accuracy is far inside the worst case (FP32 would give ~1e-7)
    assert np.median(errs) < 1e-14


def test_recip_pivot_within_one_ulp(probe):
    rng = np.random.default_rng(10)
    d = (np.exp2(rng.uniform(-120, 120, 20000)) * rng.choice([-1, 1], 20000)).astype(np.float32)
    d = np.concatenate([d, np.float32([1.0, -1.0, 3.0, 7.0, 0.1])])
    r = torch.empty(d.size, dtype=torch.float32, device="cuda")
    assert probe.probe_recip(_ptr(_dev(d)), _ptr(r), d.size) == 0
    r = r.cpu().numpy().astype(np.float64)
    exact = 1.0 / d.astype(np.float64)
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(r - exact) <= ulp)


def test_gershgorin_row_test_is_sound(probe):
    rng = np.random.default_rng(11)
    n, mats = 12, 400
    rows = []
    for k in range(mats):
        P = rng.standard_normal((n, n)).astype(np.float32) * np.float32(10.0 ** rng.uniform(-1, 3))
        # push diagonals around the Gershgorin boundary
        P[np.arange(n), np.arange(n)] = (np.sum(np.abs(P), axis=1) - np.abs(np.diag(P))
                                         + rng.uniform(-2, 2, n)).astype(np.float32)
        rows.append(P)
    P = np.concatenate(rows)
    for delta in (0.0, 1e-8, 1e-3, 0.3, 7.0):
        pas = torch.empty(P.shape[0], dtype=torch.int32, device="cuda")
        assert probe.probe_gersh(_ptr(_dev(P)), P.shape[0], n, ctypes.c_double(delta), _ptr(pas)) == 0
        pas = pas.cpu().numpy()
        dl = Fraction(delta)
        for r in range(P.shape[0]):
            i = r % n
            row = [Fraction(float(x)) for x in P[r]]
            off = sum(abs(x) for x in row) - abs(row[i])
            val = 1 + dl * (row[i] - off)
            if pas[r]:
                assert val > 0, (delta, r)
            mag = 1 + dl * (abs(row[i]) + off)
            if val > Fraction(1, 10 ** 5) * mag:
                assert pas[r], (delta, r, float(val))


def _pd_cases(rng, n, delta, count):
    """FP32 P with I + delta P of prescribed spectra, in a scaled basis:
    M = D0 (V diag(lam) V^T) D0 with D0 spread over up to 8 decades (the
    barrier-scaled diagonals), P = (M - I) / delta rounded to FP32."""
    mats = []
    for k in range(count):
        V, _ = np.linalg.qr(rng.standard_normal((n, n)))
        kind = k % 4
        lam = 10.0 ** rng.uniform(-2, 2, n)
        if kind == 1:    # indefinite: one eigenvalue slightly below zero
            lam[0] = -10.0 ** rng.uniform(-9, -3) * lam.max()
        elif kind == 2:  # PD, close to singular
            lam[0] = 10.0 ** rng.uniform(-9, -5) * lam.max()
        C = (V * lam) @ V.T
        d0 = 10.0 ** rng.uniform(0, 4 if kind == 3 else 1, n)
        M = d0[:, None] * C * d0[None, :]
        P = ((M - np.eye(n)) / delta).astype(np.float32)
        P = np.triu(P) + np.triu(P, 1).T  # exactly symmetric
        mats.append(P)
    return mats


@pytest.mark.parametrize("n", [12, 24, 48])
@pytest.mark.parametrize("tau", [0.0, 2.0 ** -15])
def test_fp32_cholesky_pd_proof(probe, n, tau):
    """With the margin tau the proof is for I + delta P - tau D (D its
    diagonal): a pass implies that matrix PD, and every matrix whose
    Jacobi-scaled smallest eigenvalue exceeds tau by a clear gap passes."""
    rng = np.random.default_rng(100 + n)
    for delta in (1e-3, 0.3, 7.0):
        mats = _pd_cases(rng, n, delta, 64)
        P = np.stack(mats)
        pas = torch.empty(len(mats), dtype=torch.int32, device="cuda")
        assert probe.probe_pdproof(_ptr(_dev(P)), len(mats), n, ctypes.c_double(delta),
                                   ctypes.c_float(tau), _ptr(pas)) == 0
        pas = pas.cpu().numpy()
        passed = 0
        for k, Pk in enumerate(mats):
            M = np.eye(n) + delta * Pk.astype(np.float64)
            Mt = M - tau * np.diag(np.diag(M))
            lam_min = np.linalg.eigvalsh(Mt).min()
            tol = 64 * n * np.finfo(np.float64).eps * np.abs(M).max()
            if pas[k]:
                # sound: a proof never passes a matrix that is not PD
                assert lam_min > -tol, (n, delta, k, lam_min)
                passed += 1
            # complete where the Jacobi-scaled spectrum is clear of tau
            d = 1.0 / np.sqrt(np.abs(np.diag(M)))
            lam_s = np.linalg.eigvalsh(d[:, None] * M * d[None, :]).min()
            if lam_s > 2e-3 + tau:
                assert pas[k], (n, delta, k, lam_s)
        assert passed >= len(mats) // 4


def test_measured_pipe_rates_are_consistent():
    """rlqr_measure_pipes (the roofline denominators): positive rates, FP32
    far above FP64 on this part, the packed f32x2 FMA at least as fast as
    the scalar one, and the TF32 tensor-core rate above the FP32 FMA rate."""
    from paper_2509_16370_b300 import rlqr
    p = rlqr.rlqr_measure_pipes()
    assert 0.0 < p["fp64_tflops"] < p["fp32_tflops"] / 10
    assert p["fp32x2_tflops"] >= 0.9 * p["fp32_tflops"]
    assert p["tf32_mma_tflops"] > p["fp32_tflops"]
