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


def make(name):
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
    names = sys.argv[1:] or list(FX.CASES)
    for n in names:
        if n not in FX.CASES:
            raise SystemExit(f"unknown fixture {n!r}; known: {', '.join(FX.CASES)}")
    if len(names) == 1:
        print(make(names[0]))
        return
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for res in pool.imap_unordered(make, names):
            print(res, flush=True)


if __name__ == "__main__":
    main()
