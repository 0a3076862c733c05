"""Reports built on converged runs of the library (GPU).

``cfb``: the Reynolds-number study of Section 4.1.2.6 (Fig. 12).  For each
Re_tau in {2e3, 4.2e3, 8e3, 2e4} and each wall scheme (HRFD with beta = 0.28,
slip-velocity bounce-back, Cai-Degrigny) a 2-D half channel with N = 20 cells
per half-width runs through lbm_run_to_convergence (the Section 4.1.1
criterion, 1e-4, per chunk of 1000 steps) and reports the bulk velocity U_b,
Re_b = 2 h U_b / nu, the computed u_tau (mean over the wall nodes), the bulk
friction coefficient C_fb = 2 (u_tau / U_b)^2 and Dean's correlation
C_fb = 0.073 Re_b^(-1/4) at the computed Re_b.  Petukhov's correlation, the
other reference of Fig. 12, is not printed in the paper and is not reported.

    python -m paper_2506_03905_gb300.reports cfb [--storage fp32|fp64] [--json FILE]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import lbm_cases as C  # noqa: E402

RE_TAU = (2000.0, 4200.0, 8000.0, 20000.0)
SCHEMES = ("wall_hrfd", "wall_bb", "wall_cai_degrigny")


def cfb_sweep(storage: str = "fp32", tol: float = 1e-4, check_every: int = 1000,
              max_steps: int = 200000):
    import paper_2506_03905_gb300 as pkg
    rows = []
    for re_tau in RE_TAU:
        for scheme in SCHEMES:
            case = C.channel_reynolds_sweep(re_tau, scheme, storage=storage)
            s = pkg.Solver(case)
            s.set_fields(*C.initial_fields(case))
            steps, res = s.run_to_convergence(tol, check_every, max_steps)
            f = s.fields(["u", "u_tau_ymin"])
            s.close()
            u_b = float(f["u"][0].mean())
            u_tau = float(f["u_tau_ymin"].mean())
            cfb = 2.0 * (u_tau / u_b) ** 2
            re_b = 2.0 * 1.0 * u_b / case.nu
            dean = C.dean_cfb(re_b)
            rows.append(dict(re_tau=re_tau, scheme=scheme, storage=storage, steps=steps,
                             residual=res, converged=bool(res < tol), u_b=u_b, re_b=re_b,
                             u_tau=u_tau, u_tau_target=C.channel_parameters(re_tau)["u_tau"],
                             cfb=cfb, cfb_dean=dean, rel_to_dean=cfb / dean - 1.0))
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("report", choices=["cfb"])
    ap.add_argument("--storage", default="fp32")
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    rows = cfb_sweep(a.storage)
    print(f"{'Re_tau':>7} {'scheme':>18} {'steps':>6} {'Re_b':>10} {'u_tau':>8} "
          f"{'C_fb':>9} {'Dean':>9} {'diff':>7}")
    for r in rows:
        print(f"{r['re_tau']:7.0f} {r['scheme']:>18} {r['steps']:6d} {r['re_b']:10.4g} "
              f"{r['u_tau']:8.5f} {r['cfb']:9.6f} {r['cfb_dean']:9.6f} {100 * r['rel_to_dean']:6.2f}%")
    if a.json:
        with open(a.json, "w") as fh:
            json.dump(rows, fh, indent=1)


if __name__ == "__main__":
    main()
