"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times.

* the 2-D half channel (D2Q9, 4 x 48, log-law bounce-back at the first node,
  BGK, SA, from rest) for its full 20,000 steps, FP64 storage, against the
  FP64 oracle;
* the 3-D channel at 256 x 128 x 128 (FP32, both wall schemes): every cell
  after 2 steps against the oracle run on the whole lattice;
* properties at full size: the benchmark's channel stays finite with mass kept
  to FP32 rounding over three times the benchmark's step count, half-way
  bounce-back conserves mass, and a fluid at rest stays exactly at rest.
"""
import numpy as np
import pytest

import lbm_cases as C
from oracle import Oracle

pytestmark = pytest.mark.gpu


def rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def test_half_channel_2d_full_20k_steps_fp64():
    import paper_2506_03905_gb300 as pkg
    case = C.half_channel_2d(storage="fp64")           # 4 x 48, 20k steps, from rest
    init = C.initial_fields(case)
    s = pkg.Solver(case)
    s.set_fields(*init)
    s.step(case.steps)
    got = s.fields(["u", "nu_t", "u_tau_ymin", "cf_ymin"])
    s.close()
    ref = Oracle(case, *init).run(case.steps).fields()
    for k in got:
        assert rel(got[k], ref[k]) < 1e-9, (k, rel(got[k], ref[k]))


@pytest.mark.parametrize("scheme,interp", [("wall_bb", "none"), ("wall_bb", "yu"),
                                           ("wall_hrfd", "none")])
def test_channel_full_size_two_steps(scheme, interp):
    import paper_2506_03905_gb300 as pkg
    case = C.channel_3d(re_tau=5200.0, scheme=scheme, interp=interp)  # 256 x 128 x 128, FP32
    init = C.initial_fields(case)
    s = pkg.Solver(case)
    s.set_fields(*init)
    s.step(2)
    names = ["u", "nu_t", "u_tau_ymin", "u_tau_ymax", "cf_ymin", "cf_ymax"]
    got = s.fields(names)
    s.close()
    ref = Oracle(case, *init).run(2).fields()
    for k in names:
        assert rel(got[k], ref[k]) < 1e-5, (k, rel(got[k], ref[k]))


def test_channel_full_size_benchmark_run_stays_finite():
    """The benchmark's channel (Yu's rule at d_w = 1/2) over three times the
    benchmark's default warm-up + timed steps: finite, every Newton converged,
    and mass kept to FP32 rounding of the stored deviations (Yu's rule at
    q = 1/2 conserves it to rounding in the FP64 oracle)."""
    import paper_2506_03905_gb300 as pkg
    case = C.channel_3d(re_tau=5200.0, scheme="wall_bb", d_w=0.5, interp="yu")
    s = pkg.Solver(case)
    s.set_fields(*C.initial_fields(case))
    d0 = s.diagnostics()
    s.step(3600)
    d1 = s.diagnostics()
    uy = np.abs(s.fields(["u"])["u"][1]).max()
    s.close()
    assert d1.nonfinite == 0 and d1.newton_failures == 0
    assert abs(d1.mass - d0.mass) / d0.mass < 2e-6
    assert uy < 1e-2 * C.channel_parameters(5200.0)["u_b"]   # no growing wall-row mode


def test_channel_full_size_half_way_mass_conservation():
    """Eq. 31 with a tangential wall velocity conserves mass; FP32 rounding of
    the stored deviations is the only drift (over 600 steps, before the
    half-way rule's wall-row oscillation has grown)."""
    import paper_2506_03905_gb300 as pkg
    case = C.channel_3d(re_tau=5200.0, scheme="wall_bb")
    s = pkg.Solver(case)
    s.set_fields(*C.initial_fields(case))
    d0 = s.diagnostics()
    s.step(600)
    d1 = s.diagnostics()
    s.close()
    assert abs(d1.mass - d0.mass) / d0.mass < 2e-6
    assert d1.nonfinite == 0 and d1.newton_failures == 0


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_channel_full_size_rest_state(storage):
    import paper_2506_03905_gb300 as pkg
    case = C.channel_3d(re_tau=5200.0, scheme="wall_hrfd", storage=storage).replace(
        force=(0.0, 0.0, 0.0), u_init=(0.0, 0.0, 0.0), perturb=0.0)
    s = pkg.Solver(case)
    s.set_fields(*C.initial_fields(case))
    s.step(10)
    f = s.fields(["u", "rho"])
    s.close()
    assert np.abs(f["u"]).max() == 0.0 and np.all(f["rho"] == case.rho0)
