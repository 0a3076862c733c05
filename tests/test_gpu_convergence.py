"""Convergence-driven runs (Section 4.1.1: converged when the relative change of
u_tau falls below 1e-4), through the C ABI."""
import numpy as np
import pytest

import lbm_cases as C
from oracle import Oracle

pytestmark = pytest.mark.gpu


def test_run_to_convergence_half_channel():
    """2-D half channel started from the bulk velocity of Dean's correlation.
    The library stops at the first 1000-step chunk whose largest relative u_tau
    change is below 1e-4; the FP64 oracle, run for the same number of steps,
    agrees on u_tau, confirms the change over the last chunk, and the converged
    u_tau is within a few per cent of the friction velocity the body force
    imposes (u_tau = Re_tau nu / h)."""
    import paper_2506_03905_gb300 as pkg
    par = C.channel_parameters(2000.0)
    case = C.half_channel_2d(storage="fp64").replace(u_init=(par["u_b"], 0.0, 0.0))
    init = C.initial_fields(case)
    s = pkg.Solver(case)
    s.set_fields(*init)
    steps, res = s.run_to_convergence(tol=1e-4, check_every=1000, max_steps=80000)
    got = s.fields(["u", "u_tau_ymin"])
    s.close()
    assert res < 1e-4 and steps % 1000 == 0 and 1000 < steps < 80000

    # the same trajectory through lbm_step
    s2 = pkg.Solver(case)
    s2.set_fields(*init)
    s2.step(steps)
    again = s2.fields(["u", "u_tau_ymin"])
    s2.close()
    assert np.array_equal(got["u"], again["u"])

    o = Oracle(case, *init).run(steps - 1000)
    ut_a = o.fields()["u_tau_ymin"]
    ut_b = o.run(1000).fields()["u_tau_ymin"]
    assert np.abs(got["u_tau_ymin"] - ut_b).max() / np.abs(ut_b).max() < 1e-9
    assert np.max(np.abs(ut_b - ut_a) / ut_b) < 1e-4
    assert abs(ut_b.mean() / par["u_tau"] - 1.0) < 0.05


def test_run_to_convergence_limits_and_errors():
    import paper_2506_03905_gb300 as pkg
    case = C.channel_3d(nx=16, ny=12, nz=2)
    s = pkg.Solver(case)
    s.set_fields(*C.initial_fields(case))
    steps, res = s.run_to_convergence(tol=1e-12, check_every=7, max_steps=20)
    assert steps == 20 and res >= 1e-12          # chunks of 7, 7 and 6 steps
    n0 = s.kernel_launches()
    with pytest.raises(pkg.LbmError):
        s.run_to_convergence(tol=0.0)
    with pytest.raises(pkg.LbmError):
        s.run_to_convergence(check_every=0)
    assert s.kernel_launches() == n0
    s.close()
    periodic = case.replace(bcs={"ymin": C.BC("periodic"), "ymax": C.BC("periodic")})
    s = pkg.Solver(periodic)
    s.set_fields(*C.initial_fields(periodic))
    with pytest.raises(pkg.LbmError):
        s.run_to_convergence()
    s.close()
