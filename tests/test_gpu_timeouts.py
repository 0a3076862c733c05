"""Bounded device-side waits that run out, on the GPU, without a fault or a hang.

Every wait of the library's kernels polls a bounded number of times and then
gives up, records the failure and leaves the kernel; the host reports
LBM_ETIMEOUT.  A test-only limit of 0 polls makes the waits give up at once:

* the batch kernel: a warp waiting for an earlier item of its instance gives up,
  every warp leaves at its next ticket or wait, lbm_batch_wait reports
  LBM_ETIMEOUT; with the default limit restored and the states set again the
  same batch then computes what single instances compute;
* a launch that gave up is reported even when the host enqueues another,
  successful launch before it looks (each launch's failure record has its own
  host copy);
* the TMA-staged inner-row kernel: every block gives up on its first tile,
  waits (with the default bound) for its copies in flight and leaves;
  lbm_fields reports LBM_ETIMEOUT, and the context is usable again after a
  new lbm_set_fields.
"""
import numpy as np
import pytest

import lbm_cases as C

pytestmark = pytest.mark.gpu

DEFAULT_POLLS = 1 << 24


def rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def test_batch_wait_runs_out_and_the_batch_recovers():
    import paper_2506_03905_gb300 as pkg
    from test_gpu_batch import mixed_cases, solvers
    cases = mixed_cases()
    ss = solvers(cases)
    b = pkg.lbm_batch_create([s.ctx for s in ss])
    pkg.lbm_batch_set_mode(b, 0)      # the persistent kernel: the mode with device-side waits
    pkg.lbm_batch_tune(b)
    assert pkg.lbm_batch_info(b)["mode"] == 0
    assert pkg.lbm_batch_wait(b) == pkg.LBM_OK
    pkg.lbm_batch_set_wait_limit(b, 0)
    pkg.lbm_batch_step(b, 3)          # enqueued; the failure is reported by the wait
    assert pkg.lbm_batch_wait(b) == pkg.LBM_ETIMEOUT
    assert "gave up" in pkg.lbm_batch_last_error(b)
    assert pkg.lbm_batch_wait(b) == pkg.LBM_OK    # reported once
    # recovery: default limit, fresh states, then the batch against single instances
    pkg.lbm_batch_set_wait_limit(b, DEFAULT_POLLS)
    for s, c in zip(ss, cases):
        s.set_fields(*C.initial_fields(c))
    nsteps = 7
    pkg.lbm_batch_step(b, nsteps)
    assert pkg.lbm_batch_wait(b) == pkg.LBM_OK
    got = [s.fields(["u"])["u"] for s in ss]
    pkg.lbm_batch_destroy(b)
    for s in ss:
        s.close()
    single = solvers(cases)
    for s in single:
        s.step(nsteps)
    ref = [s.fields(["u"])["u"] for s in single]
    for s in single:
        s.close()
    for c, g, r in zip(cases, got, ref):
        assert rel(g, r) < 1e-6, c.name


def test_batch_timeout_is_reported_after_a_later_launch():
    import paper_2506_03905_gb300 as pkg
    from test_gpu_batch import mixed_cases, solvers
    cases = mixed_cases()
    ss = solvers(cases)
    b = pkg.lbm_batch_create([s.ctx for s in ss])
    pkg.lbm_batch_set_mode(b, 0)
    pkg.lbm_batch_tune(b)
    assert pkg.lbm_batch_wait(b) == pkg.LBM_OK
    pkg.lbm_batch_set_wait_limit(b, 0)
    pkg.lbm_batch_step(b, 3)          # gives up
    pkg.lbm_batch_set_wait_limit(b, DEFAULT_POLLS)
    # enqueued before the host has looked at the first launch, if that one is
    # still running; otherwise this call already reports it
    try:
        pkg.lbm_batch_step(b, 3)
        st = pkg.lbm_batch_wait(b)
    except pkg.LbmError as exc:
        st = exc.status
    assert st == pkg.LBM_ETIMEOUT
    assert pkg.lbm_batch_wait(b) == pkg.LBM_OK
    pkg.lbm_batch_destroy(b)
    for s in ss:
        s.close()


def test_tma_tile_wait_runs_out_and_the_context_recovers():
    import paper_2506_03905_gb300 as pkg
    case = C.channel_3d(re_tau=5200.0, scheme="wall_bb", nx=64, ny=34, nz=12, seed=2)
    s = pkg.Solver(case, tma_staging=True)
    s.set_fields(*C.initial_fields(case))
    pkg.lbm_set_wait_limit(s.ctx, 0)
    s.step(2)
    s.fields(["u"], check=False)
    assert s.last_status == pkg.LBM_ETIMEOUT, pkg.lbm_last_error(s.ctx)
    pkg.lbm_set_wait_limit(s.ctx, DEFAULT_POLLS)
    s.set_fields(*C.initial_fields(case))
    s.step(5)
    got = s.fields(["u", "nu_t"])
    s.close()
    ref_s = pkg.Solver(case)
    ref_s.set_fields(*C.initial_fields(case))
    ref_s.step(5)
    ref = ref_s.fields(["u", "nu_t"])
    ref_s.close()
    for k in got:
        assert rel(got[k], ref[k]) < 1e-6, k
