"""Storage precision on the flat-plate crop: FP32 / FP16 / BF16 shifted
populations (FP32 arithmetic, FP64 u_tau Newton and sums) against the FP64
oracle on the same seeded input.

Workload: the D3Q19 zero-pressure-gradient plate on 512 x 128 x 4 cells at
Delta = 4e-3 m (the plate geometry of Section 4.2.1, x in [-0.2, 1.848] m,
Zou-He inlet, zero-gradient outlet, free-stream top, symmetry before the
leading edge), regularized collision, slip-velocity bounce-back and HRFD walls.

Reported per storage: max relative error of C_f(x) over the plate, the
integrated error eps = int |C_f - C_f,ref| dx / int C_f,ref dx over
x in [1, 1.8] (the error measure of Section 4.2.2, trapezoid rule, here
against the oracle), the max error of u+ = u / u_tau,ref over the first
three rows above the plate, and of nu_t relative to its maximum.  The bar is
C_f error <= 1 % for the 16-bit storages and <= 1e-5 for FP32.
"""
import json
import os

import numpy as np
import pytest

import lbm_cases as C
from oracle import Oracle

pytestmark = pytest.mark.gpu

NSTEPS = 200


def _errors(case, got, ref, x):
    plate = x >= 0.0
    cf_g, cf_r = got["cf_ymin"][:, plate], ref["cf_ymin"][:, plate]
    cf_err = float(np.abs(cf_g - cf_r).max() / np.abs(cf_r).max())
    win = (x >= 1.0) & (x <= 1.8)
    g = got["cf_ymin"][:, win].mean(0)
    r = ref["cf_ymin"][:, win].mean(0)
    xs = x[win]
    trap = getattr(np, "trapezoid", None) or np.trapz
    eps = float(trap(np.abs(g - r), xs) / trap(r, xs))
    ut = ref["u_tau_ymin"][:, plate]
    up_g = got["u"][0][:, :3, plate] / ut[:, None, :]
    up_r = ref["u"][0][:, :3, plate] / ut[:, None, :]
    uplus_err = float(np.abs(up_g - up_r).max())
    nut_err = float(np.abs(got["nu_t"] - ref["nu_t"]).max() / np.abs(ref["nu_t"]).max())
    return dict(cf_max_rel=cf_err, eps_cf=eps, uplus_max_abs=uplus_err, nut_rel=nut_err,
                uplus_ref_max=float(np.abs(up_r).max()))


@pytest.mark.parametrize("scheme", ["wall_bb", "wall_hrfd"])
def test_plate_storage_precision(scheme):
    import paper_2506_03905_gb300 as pkg
    base = C.flat_plate_3d(nx=512, ny=128, nz=4, dx=4e-3, scheme=scheme, collision="regularized")
    init = C.initial_fields(base)
    o = Oracle(base, *init).run(NSTEPS)
    ref = o.fields()
    x = o.xc
    names = ["u", "nu_t", "u_tau_ymin", "cf_ymin"]
    report = {}
    for storage in ("fp32", "fp16", "bf16"):
        case = base.replace(storage=storage)
        s = pkg.Solver(case)
        s.set_fields(*init)
        s.step(NSTEPS)
        got = s.fields(names)
        s.close()
        report[storage] = _errors(case, got, ref, x)
    out = os.environ.get("LBM_REPORT_DIR")   # optional: keep the error report as JSON
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, f"precision_plate_{scheme}.json"), "w") as fh:
            json.dump(dict(case=base.name, steps=NSTEPS, errors=report), fh, indent=1)
    assert report["fp32"]["cf_max_rel"] < 1e-5, report
    for st in ("fp16", "bf16"):
        assert report[st]["cf_max_rel"] < 1e-2, (st, report)
