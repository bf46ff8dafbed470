"""CPU checks of the C ABI library: it loads, exports every entry point that
include/rlqr.h, include/rlqr_ipm.h and include/rlqr_mlp.h declare, and validates arguments on the
host (no GPU call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = "".join(open(os.path.join(ROOT, "include", h)).read() for h in ("rlqr.h", "rlqr_ipm.h", "rlqr_mlp.h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(rlqr_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_abi():
    names = _declared()
    for want in ("rlqr_factor", "rlqr_solve", "rlqr_residual", "rlqr_solve_batched",
                 "rlqr_workspace_bytes", "rlqr_batched_workspace_bytes"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2509_16370_b300 import rlqr
    lib = ctypes.CDLL(rlqr.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(rlqr.EXPORTED) <= set(_declared())
    from paper_2509_16370_b300 import ipm
    assert set(ipm.EXPORTED) <= set(_declared())
    from paper_2509_16370_b300 import mlp
    assert set(mlp.EXPORTED) <= set(_declared())


def test_ipm_host_side_validation_and_sizes():
    from paper_2509_16370_b300 import ipm
    m, o = ipm.make_model(), ipm.make_ipm_opts()
    a = ipm.rlqr_ipm_workspace_bytes(16, m, o)
    b = ipm.rlqr_ipm_workspace_bytes(32, m, o)
    assert 0 < a < b and a % 256 == 0
    assert ipm.rlqr_ipm_workspace_bytes(0, m, o) == 0
    assert ipm.rlqr_ipm_workspace_bytes(16, ipm.make_model(N=0), o) == 0
    assert ipm.rlqr_ipm_workspace_bytes(16, ipm.make_model(N=5000), o) == 0
    assert ipm.rlqr_ipm_workspace_bytes(16, m, ipm.make_ipm_opts(tau=1.0)) == 0
    assert ipm.rlqr_ipm_workspace_bytes(16, m, ipm.make_ipm_opts(hessian=3)) == 0
    assert ipm.rlqr_ipm_workspace_bytes(16, m, ipm.make_ipm_opts(ls_steps=0)) == 0
    st = ipm.rlqr_ipm_state()
    code = ipm.lib.rlqr_ipm_iterate(16, ctypes.byref(m), ctypes.byref(o), None, None,
                                    ctypes.byref(st), None, 0, None, None)
    assert code == 2   # RLQR_ERR_ARG before any device work


def test_host_side_validation_and_sizes():
    from paper_2509_16370_b300 import rlqr
    o = rlqr.make_opts(rlqr.RLQR_FP64)
    assert rlqr.rlqr_workspace_bytes(0, 4, 2, o) == 0
    assert rlqr.rlqr_workspace_bytes(8, 0, 2, o) == 0
    assert rlqr.rlqr_workspace_bytes(8, 4, 0, o) == 0
    assert rlqr.rlqr_workspace_bytes(8, 49, 2, o) == 0      # above the largest kernel bucket
    a = rlqr.rlqr_workspace_bytes(64, 4, 2, o)
    om = rlqr.make_opts(rlqr.RLQR_MIXED)
    b = rlqr.rlqr_workspace_bytes(64, 4, 2, om)
    assert a > 0 and b > 0 and a % 256 == 0 and b % 256 == 0
    # the scan path adds its chunk arrays; AUTO sizes for the scan from N = 4096 on
    seq = rlqr.make_opts(rlqr.RLQR_FP64, algo=rlqr.RLQR_ALGO_SEQ)
    scan = rlqr.make_opts(rlqr.RLQR_FP64, algo=rlqr.RLQR_ALGO_SCAN)
    assert rlqr.rlqr_workspace_bytes(64, 4, 2, scan) > rlqr.rlqr_workspace_bytes(64, 4, 2, seq)
    assert rlqr.rlqr_workspace_bytes(64, 4, 2, o) == rlqr.rlqr_workspace_bytes(64, 4, 2, seq)
    assert (rlqr.rlqr_workspace_bytes(4096, 32, 8, o) ==
            rlqr.rlqr_workspace_bytes(4096, 32, 8, scan))
    assert (rlqr.rlqr_workspace_bytes(4096, 5, 2, o) ==
            rlqr.rlqr_workspace_bytes(4096, 5, 2, seq))   # no scan kernel for (5, 2)
    bad = rlqr.make_opts(rlqr.RLQR_FP64, tol=-1.0)
    assert rlqr.rlqr_workspace_bytes(8, 4, 2, bad) == 0
    # invalid problem: rejected before any device work
    ps = rlqr.rlqr_problem()
    ps.N, ps.nx, ps.nu = 0, 4, 2
    code = rlqr.lib.rlqr_factor(ctypes.byref(ps), ctypes.byref(o), None, 0, None, None, None)
    assert code == rlqr.RLQR_ERR_ARG
    assert rlqr.lib.rlqr_solve_batched(None, ctypes.byref(o), None, 0, None, None, None,
                                       None) == rlqr.RLQR_ERR_ARG
    assert "rlqr-b300" in rlqr.version()
    assert rlqr.lib.rlqr_status_string(rlqr.RLQR_ERR_SINGULAR).decode().startswith("zero")
