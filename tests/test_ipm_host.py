"""Host-side checks of the IPM (CPU): the constants of the method agree
between the oracle's Options and the binding's defaults (the parity tests
compare the two sides with them), the problem data come from the one
workload definition, and the workload's inputs are reproducible."""
import numpy as np

import oracle.ipm as O
from paper_2509_16370_b300 import inputs
from paper_2509_16370_b300 import ipm as G


def test_method_constants_agree():
    op, g = O.Options(), G.make_ipm_opts()
    for k in ("max_iter", "tol", "eta", "mu0", "mu_min", "kappa_mu", "tau", "armijo", "ls_steps",
              "rho_first", "rho_grow", "rho_shrink", "rho_min", "rho_max", "kappa_sigma",
              "s_min"):
        assert getattr(g, k) == getattr(op, k), k
    assert g.hessian == G.RLQR_IPM_HESS_EXACT_FP32 and op.exact_hessian


def test_problem_data_agree():
    md, gm = O.Model(), G.make_model()
    for k in ("N", "dt", "m0", "m1", "m2", "l1", "l2", "grav", "u_max", "p_max", "wu"):
        assert getattr(gm, k) == getattr(md, k) == inputs.CDP_MODEL[k], k
    assert list(gm.wx) == list(md.wx) == list(inputs.CDP_MODEL["wx"])
    assert list(gm.wf) == list(md.wf) == list(inputs.CDP_MODEL["wf"])


def test_workload_inputs_are_reproducible():
    a0, ag = inputs.workload5(16, 100)
    b0, bg = inputs.workload5(16, 100)
    np.testing.assert_array_equal(a0, b0)
    np.testing.assert_array_equal(ag, bg)
    x0, xg = inputs.workload5_instance(107)
    np.testing.assert_array_equal(a0[7], x0)
    assert np.all(np.abs(a0[:, 1:3]) <= np.pi) and np.all(a0[:, [0, 3, 4, 5]] == 0)
    assert np.all(np.abs(ag[:, 0]) <= 1) and np.all(ag[:, 1:] == 0)
