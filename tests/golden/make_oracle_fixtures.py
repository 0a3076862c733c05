#!/usr/bin/env python3
"""Write the oracle fixtures of tests/fixture_cases.py into tests/golden/oracle/.

Runs the FP64 oracle (``oracle/``) on the seeded inputs of ``lbm_cases`` and
stores the reduced results; it imports nothing from the CUDA package.  Usage:

    python tests/golden/make_oracle_fixtures.py            # every fixture
    python tests/golden/make_oracle_fixtures.py NAME ...   # selected ones

Each fixture takes minutes to an hour of one CPU core; names run in parallel
processes when several are given.
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import lbm_cases as C  # noqa: E402
import fixture_cases as FX  # noqa: E402
from oracle import Oracle  # noqa: E402


def bulk_friction(case, o):
    """U_b (mean of u_x over the half channel), mean wall u_tau and
    C_fb = 2 (u_tau / U_b)^2 of an oracle state (Section 4.1.2.6)."""
    f = o.fields()
    u_b = float(f["u"][0].mean())
    u_tau = float(f["u_tau_ymin"].mean())
    return u_b, u_tau, 2.0 * (u_tau / u_b) ** 2


def make_cfb(name):
    """Run the oracle until the Section 4.1.1 criterion holds for a chunk of
    CFB_CHECK steps: max over wall nodes of |u_tau - u_tau_prev| / u_tau < CFB_TOL,
    the first reference being the initial state's u_tau (zero)."""
    case = FX.cfb_case(name)
    t0 = time.time()
    o = Oracle(case, *C.initial_fields(case))
    prev = o.utau["ymin"].copy()
    steps, res = 0, np.inf
    while steps < FX.CFB_MAX:
        o.run(FX.CFB_CHECK)
        steps += FX.CFB_CHECK
        ut = o.utau["ymin"]
        pos = ut > 0
        res = float(np.max(np.abs(ut[pos] - prev[pos]) / ut[pos])) if pos.any() else np.inf
        prev = ut.copy()
        if res < FX.CFB_TOL:
            break
    u_b, u_tau, cfb = bulk_friction(case, o)
    re_b = u_b * 2.0 / case.nu                     # Re_b = U_b 2h / nu, h = 1 m
    meta = dict(signature=FX.case_signature(case), steps=steps, residual=res, u_b=u_b,
                u_tau=u_tau, cfb=cfb, re_b=re_b, case=case.name,
                seconds=round(time.time() - t0, 1))
    os.makedirs(FX.FIXDIR, exist_ok=True)
    tmp = FX.path(name) + ".tmp.npz"
    np.savez_compressed(tmp, meta=np.array(json.dumps(meta)))
    os.replace(tmp, FX.path(name))
    return name, meta["seconds"]


def make(name):
    if name in FX.CFB_CASES:
        return make_cfb(name)
    factory, steps = FX.CASES[name]
    case = factory()
    t0 = time.time()
    o = Oracle(case, *C.initial_fields(case)).run(steps)
    fields = o.fields()
    red = FX.reduce_fields(case, fields)
    meta = dict(signature=FX.case_signature(case), steps=steps, case=case.name,
                mass=o.mass(), momentum=[float(v) for v in o.momentum()],
                seconds=round(time.time() - t0, 1))
    os.makedirs(FX.FIXDIR, exist_ok=True)
    tmp = FX.path(name) + ".tmp.npz"
    np.savez_compressed(tmp, meta=np.array(json.dumps(meta)), **red)
    os.replace(tmp, FX.path(name))
    return name, meta["seconds"]


def main():
    known = list(FX.CASES) + list(FX.CFB_CASES)
    names = sys.argv[1:] or known
    for n in names:
        if n not in known:
            raise SystemExit(f"unknown fixture {n!r}; known: {', '.join(known)}")
    if len(names) == 1:
        print(make(names[0]))
        return
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for res in pool.imap_unordered(make, names):
            print(res, flush=True)


if __name__ == "__main__":
    main()
