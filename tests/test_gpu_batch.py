"""Batched sweeps: many instances advanced together, by one persistent
cooperative launch (mode 0) or by per-step multi-instance launches (mode 1).

In either mode the batch must give what each instance gives when stepped alone
(same arithmetic; compiled in different kernels, so agreement is to rounding),
and the instances must still match the FP64 oracle.
"""
import numpy as np
import pytest

import lbm_cases as C
from oracle import Oracle

pytestmark = pytest.mark.gpu


def rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def mixed_cases(storage="fp32"):
    return [
        C.channel_3d(re_tau=2000.0, scheme="wall_bb", nx=4, ny=24, nz=1, seed=1,
                     storage=storage).replace(lattice="D2Q9"),
        C.channel_3d(re_tau=5200.0, scheme="wall_hrfd", nx=20, ny=16, nz=4, seed=2, storage=storage),
        C.flat_plate_3d(nx=48, ny=12, nz=2, dx=4e-2, scheme="wall_bb", storage=storage),
        C.flat_plate_3d(nx=40, ny=10, nz=1, dx=5e-2, scheme="wall_hrfd",
                        storage=storage).replace(lattice="D2Q9"),
        C.channel_3d(re_tau=1000.0, scheme="wall_bb", nx=36, ny=18, nz=3, seed=4,
                     collision="regularized", storage=storage),
    ]


def solvers(cases):
    import paper_2506_03905_gb300 as pkg
    out = []
    for c in cases:
        s = pkg.Solver(c)
        s.set_fields(*C.initial_fields(c))
        out.append(s)
    return out


FIELDS = ["u", "nu_t", "u_tau_ymin"]


# lbm_batch_tune: mode 0's 2 block sizes x 3 tiles and mode 1, each 1 warm-up + 3 timed steps
TUNE_STEPS = 7 * 4


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_matches_single_instances_and_oracle(mode):
    import paper_2506_03905_gb300 as pkg
    cases = mixed_cases()
    nsteps = 40
    single = solvers(cases)
    for s in single:
        s.step(nsteps)
    ref = [s.fields(FIELDS) for s in single]
    for s in single:
        s.close()
    batch_s = solvers(cases)
    b = pkg.lbm_batch_create([s.ctx for s in batch_s])
    pkg.lbm_batch_set_mode(b, mode)
    threads, tile = pkg.lbm_batch_tune(b)          # tuning advances every instance
    assert threads in (128, 256) and tile in (64, 256, 1024)   # cells per warp item
    assert batch_s[0].steps_done() == TUNE_STEPS
    assert pkg.lbm_batch_info(b)["mode"] == mode
    pkg.lbm_batch_step(b, nsteps - TUNE_STEPS - 5)
    pkg.lbm_batch_step(b, 5)
    got = [s.fields(FIELDS) for s in batch_s]
    pkg.lbm_batch_destroy(b)
    for s in batch_s:
        s.close()
    for c, g, r in zip(cases, got, ref):
        for k in FIELDS:
            assert rel(g[k], r[k]) < 1e-6, (c.name, k, rel(g[k], r[k]))
    # and each instance against the FP64 oracle
    for c, g in zip(cases, got):
        o = Oracle(c, *C.initial_fields(c)).run(nsteps).fields()
        for k in FIELDS:
            assert rel(g[k], o[k]) < 1e-5, (c.name, k, rel(g[k], o[k]))


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_interleaved_with_single_steps(mode):
    """Stepping the members on their own between batch launches keeps every
    instance's buffer parity right."""
    import paper_2506_03905_gb300 as pkg
    cases = mixed_cases()[:3]
    nsteps = TUNE_STEPS + 1 + 5 + 33     # 33: a captured chunk of 32 steps plus one direct step
    a = solvers(cases)
    for s in a:
        s.step(nsteps)
    ref = [s.fields(["u"])["u"] for s in a]
    for s in a:
        s.close()
    bs = solvers(cases)
    b = pkg.lbm_batch_create([s.ctx for s in bs])
    pkg.lbm_batch_set_mode(b, mode)
    pkg.lbm_batch_tune(b)
    for s in bs:
        s.step(1)                  # odd number of single steps: parity flips
    pkg.lbm_batch_step(b, 5)
    pkg.lbm_batch_step(b, 33)
    got = [s.fields(["u"])["u"] for s in bs]
    pkg.lbm_batch_destroy(b)
    for s in bs:
        s.close()
    for g, r in zip(got, ref):
        assert rel(g, r) < 1e-6


def test_batch_rejects_mixed_storage():
    import paper_2506_03905_gb300 as pkg
    cs = [mixed_cases("fp32")[1], mixed_cases("fp16")[1]]
    ss = solvers(cs)
    with pytest.raises(pkg.LbmError):
        pkg.lbm_batch_create([s.ctx for s in ss])
    for s in ss:
        s.close()


def test_batch_fp16_storage_runs():
    import paper_2506_03905_gb300 as pkg
    cases = mixed_cases("fp16")
    ss = solvers(cases)
    b = pkg.lbm_batch_create([s.ctx for s in ss])
    pkg.lbm_batch_step(b, 30)
    for s, c in zip(ss, cases):
        f = s.fields(["u", "rho"])
        assert np.isfinite(f["u"]).all()
        assert abs(f["rho"].mean() / c.rho0 - 1.0) < 1e-2
    pkg.lbm_batch_destroy(b)
    for s in ss:
        s.close()
