#!/usr/bin/env python3
"""Throughput benchmark of the GB300 LBM-RANS step (MLUPS and HBM roofline).

Workload (N = 1): the 3-D D3Q19 turbulent channel in FP32 storage,
256 x 128 x 128 cells, periodic in x and z, slip-velocity bounce-back walls
(Eq. 35, with Yu's rule of Eq. 37 at d_w = 1/2) on both y faces,
Re_tau = 5200, SA turbulence model, initial u_x = U_b (1 +/- 1 %) seeded and
nu_tilde = max(3 nu, kappa u_tau d).  A step is one full pass of the method:
the wall pre-pass, the wall rows and the fused SA + stream + collide kernel
on the inner rows (three launches).  The population buffers (2 x 319 MB) are
larger than the 129 MB L2, so no flush is needed between steps.

Extra keys report the HRFD and Cai-Degrigny walls, FP16/BF16 shifted
storage, the 2048 x 512 x 8 flat plate and the 96-instance batched sweep on
the same GPU.  ``--impl reference`` times the FP64 CPU oracle, one
single-threaded copy per host core, on bounded crops of the same workload;
``cpu_baseline`` in the main line is the same on 64 x 128 x 8 crops plus one
copy alone.  ``--profile-case`` and ``--profile-batch`` are short runs for
ncu.

Multi-GPU: one process per GPU (torchrun); every rank advances its own
replica of the workload (weak scaling, no data-path collective); the timed
region is bracketed by a barrier and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
if "reference" in sys.argv:
    # each oracle copy of the CPU reference arm runs on one core: one numpy thread
    for _k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_k] = "1"

import numpy as np  # noqa: E402

import lbm_cases as C  # noqa: E402

METRIC = "MLUPS and % of HBM roofline: FP32 vs FP16-storage vs batched, at C_f err ≤1%"
# slip-velocity bounce-back with Yu's rule at the half-way position: plain
# half-way bounce-back (Eq. 31) develops a growing wall-row oscillation on this
# 3-D channel (in FP64 as in FP32), which Yu's rule damps
WORKLOAD = dict(re_tau=5200.0, scheme="wall_bb", nx=256, ny=128, nz=128, seed=0, d_w=0.5,
                interp="yu")
# algorithmic bytes per cell per step: read + write every population once,
# read + write nu_tilde once (velocity and nu_t are recomputable, the wall
# distance is analytic)
ALG_BYTES = {("D3Q19", "fp32"): 160, ("D3Q19", "fp16"): 84, ("D3Q19", "bf16"): 84,
             ("D3Q19", "fp64"): 320, ("D2Q9", "fp32"): 80, ("D2Q9", "fp16"): 44,
             ("D2Q9", "bf16"): 44, ("D2Q9", "fp64"): 160}
KERNEL_SOURCES = ["paper_2506_03905_gb300/csrc/lbm_kernels.cuh",
                  "paper_2506_03905_gb300/csrc/lbm_device.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(case_key: str):
    """dram bytes per launch of the bulk kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "k_bulk_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    entry = d.get(case_key)
    if not entry or entry.get("kernel_hash") != kernel_hash():
        return None
    return entry.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.proc = None
        self.index = index
        self.path = os.path.join(tempfile.gettempdir(),
                                 f"lbm_bench_clocks_{os.getpid()}_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self._wait_lines(1, 5.0)     # nvidia-smi needs a moment before its first sample

    def _lines(self) -> int:
        try:
            with open(self.path) as fh:
                return sum(1 for _ in fh)
        except OSError:
            return 0

    def _wait_lines(self, n: int, limit_s: float):
        t0 = time.perf_counter()
        while (self.proc is not None and self.proc.poll() is None and self._lines() < n
               and time.perf_counter() - t0 < limit_s):
            time.sleep(0.005)

    def stop(self):
        if self.proc is None:
            return None
        # a timed region shorter than the 20 ms sampling period may fall between two
        # samples: keep the sampler for one more, the one closest after the region
        self._wait_lines(self._lines() + 1, 1.0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_case(pkg, case, steps, warmup, torch):
    """Device-resident timing (CUDA events on the solver's stream) and the
    per-kernel durations of the same number of steps."""
    s = pkg.Solver(case)
    s.set_fields(*C.initial_fields(case))
    s.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    bulk_ms, wall_ms = s.step_timed(steps)
    d = s.diagnostics()
    s.close()
    return ms, bulk_ms / steps, wall_ms / steps, d


def run_ours(args):
    import torch
    import paper_2506_03905_gb300 as pkg

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    pkg.lib()
    case = C.channel_3d(**WORKLOAD, storage="fp32")
    peak, peak_kind = measured_peaks()

    # ---- headline: device-resident FP32 bounce-back channel
    s = pkg.Solver(case)
    s.set_fields(*C.initial_fields(case))
    s.step(args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n_launch0 = s.kernel_launches()
    e0.record(s.stream)
    s.step(args.steps)
    e1.record(s.stream)
    n_launches = s.kernel_launches() - n_launch0
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    # per-kernel durations over the same number of steps (events around each launch)
    bulk_ms, wall_ms, inner_ms = s.step_timed3(args.steps)
    diag = s.diagnostics()
    s.close()
    cells = case.cells
    value = cells * args.steps * world / (ms * 1e-3) / 1e6
    bulk_avg = bulk_ms / args.steps
    # the dominant kernel: the inner rows (face-free, two cells per thread),
    # nx * (ny - 2) * nz cells per launch, timed alone by CUDA events
    inner_avg = inner_ms / args.steps
    inner_cells = case.nx * (case.ny - 2) * case.nz
    alg = ALG_BYTES[(case.lattice, case.storage)] * inner_cells
    achieved = alg / (inner_avg * 1e-3) / 1e9
    traffic = ncu_traffic("channel_3d_Re5200_wall_bb_256x128x128_fp32")

    # ---- end to end through the C ABI with pinned host buffers
    rho, u, nut = C.initial_fields(case)
    pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
    h_rho, h_u, h_nut = pin(rho), pin(u), pin(nut)
    h_out_u = torch.empty(u.shape, dtype=torch.float64).pin_memory()
    h_out_nut = torch.empty(nut.shape, dtype=torch.float64).pin_memory()
    s = pkg.Solver(case)
    s.set_fields(rho, u, nut)
    s.step(2)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    pkg.lbm_set_fields(s.ctx, h_rho.data_ptr(), h_u.data_ptr(), h_nut.data_ptr(), False)
    s.step(args.steps)
    st = pkg.lbm_fields(s.ctx, pkg.FIELD["u"] | pkg.FIELD["nu_t"],
                       [h_out_u.data_ptr(), h_out_nut.data_ptr()], False)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    s.close()
    h2d = (rho.nbytes + u.nbytes + nut.nbytes) / args.steps
    d2h = (u.nbytes + nut.nbytes) / args.steps
    e2e = cells * args.steps * world / e2e_s / 1e6

    # ---- variants on the same GPU (rank 0 only, short)
    variants = {}
    if world == 1 and not args.no_variants:
        # the channel variants under the headline's own step counts (the wall-law
        # Newton costs most in the early transient); the plates over 100 steps
        csteps, cwarm = args.steps, args.warmup
        vsteps = max(10, min(args.steps, 100))
        for label, kw in [("fp32_hrfd", dict(scheme="wall_hrfd", storage="fp32")),
                          ("fp32_cai", dict(scheme="wall_cai_degrigny", storage="fp32")),
                          ("fp16_bb", dict(storage="fp16")), ("bf16_bb", dict(storage="bf16")),
                          ("fp16_hrfd", dict(scheme="wall_hrfd", storage="fp16"))]:
            wk = dict(WORKLOAD)
            wk.update({k: v for k, v in kw.items() if k != "storage"})
            if wk["scheme"] != "wall_bb":
                wk["interp"] = "none"        # interpolation applies to bounce-back walls
            vc = C.channel_3d(**wk, storage=kw["storage"])
            vms, vbulk, vwall, vd = time_case(pkg, vc, csteps, cwarm, torch)
            vb = ALG_BYTES[(vc.lattice, vc.storage)] * vc.cells
            variants[label] = {
                "mlups": round(vc.cells * csteps / (vms * 1e-3) / 1e6, 1), "steps": csteps,
                "bulk_ms": round(vbulk, 4), "wall_ms": round(vwall, 4),
                "alg_bytes_per_cell": ALG_BYTES[(vc.lattice, vc.storage)],
                "bulk_frac_of_hbm": round(vb / (vbulk * 1e-3) / 1e9 / peak, 4),
                "nonfinite": int(vd.nonfinite)}
        # the flat-plate workload at full size (2048 x 512 x 8, regularized collision)
        for label, scheme in [("plate_fp32_bb", "wall_bb"), ("plate_fp32_hrfd", "wall_hrfd")]:
            pc = C.flat_plate_3d(scheme=scheme)
            pms, pbulk, pwall, pd = time_case(pkg, pc, vsteps, 3, torch)
            pb = ALG_BYTES[(pc.lattice, pc.storage)] * pc.cells
            variants[label] = {
                "mlups": round(pc.cells * vsteps / (pms * 1e-3) / 1e6, 1),
                "bulk_ms": round(pbulk, 4), "wall_ms": round(pwall, 4),
                "alg_bytes_per_cell": ALG_BYTES[(pc.lattice, pc.storage)],
                "bulk_frac_of_hbm": round(pb / (pbulk * 1e-3) / 1e9 / peak, 4),
                "nonfinite": int(pd.nonfinite)}
        bsteps = max(10, min(args.steps, 300))   # the sweep's steps are short: 300 for a stable figure
        for storage in ("fp32", "fp16"):
            try:
                variants.update(batched_variant(pkg, torch, bsteps, storage=storage))
            except Exception as exc:  # the batched path reports its own status
                variants[f"batched_{storage}"] = {"unavailable": str(exc)[:200]}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "channel_3d_D3Q19_256x128x128_fp32_Re5200_slip_bounce_back_yu",
                   "lattice": "D3Q19", "nx": 256, "ny": 128, "nz": 128, "storage": "fp32",
                   "collision": "bgk",
                   "walls": "slip-velocity bounce-back (Eq. 35) with Yu's rule (Eq. 37) at "
                            "d_w = 1/2, both y faces",
                   "init": "u_x = U_b (1 +/- 1 %) seeded, nu_tilde = max(3 nu, kappa u_tau d)",
                   "turbulence": "Spalart-Allmaras", "cells": cells,
                   "l2": "inputs larger than L2 (2 x 319 MB population buffers)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": "k_bulk2<19, fp32> (inner rows, two cells per thread)",
                     "cells_per_launch": inner_cells,
                     "alg_bytes_per_cell": ALG_BYTES[(case.lattice, case.storage)],
                     "kernel_ms": round(inner_avg, 4), "bulk_rows_ms": round(bulk_avg, 4),
                     "wall_pass_ms": round(wall_ms / args.steps, 4)},
        "e2e": {"value": round(e2e, 1), "unit": "MLUPS", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "status": int(st),
                # one FP64 field upload and one read-back per run of this many steps
                "steps_per_transfer": args.steps},
        "gpu_launches": int(n_launches),
        **({"error": "non-finite state after the timed steps"} if diag.nonfinite else {}),
        "clocks": clk,
        "diagnostics": {"mass": diag.mass, "nonfinite": int(diag.nonfinite),
                        "mean_u_tau": list(diag.mean_u_tau)},
        "variants": variants,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def batched_variant(pkg, torch, steps, rank=0, world=1, storage="fp32"):
    cases = C.batched_sweep(96, storage=storage)
    if world > 1:   # instances are independent: each rank advances its own shard
        mine = C.shard_instances([c.cells for c in cases], world, rank)
        cases = [cases[i] for i in mine]
    solvers = []
    for c in cases:
        s = pkg.Solver(c)
        s.set_fields(*C.initial_fields(c))
        solvers.append(s)
    total = sum(c.cells for c in cases)
    out = {}
    # per-case sequential runs through lbm_step: every instance of the sweep is
    # below the size at which steps of lattices with walls are launched directly,
    # so each replays its captured two-step graphs
    for s in solvers:
        s.step(steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in solvers:
        s.step(steps)
    torch.cuda.synchronize()
    seq = time.perf_counter() - t0
    out[f"per_case_{storage}"] = {"mlups": round(total * steps / seq / 1e6, 1),
                                  "instances": len(cases), "cells": total}
    b = pkg.lbm_batch_create([s.ctx for s in solvers])
    try:
        # the first call autotunes; a call with a new step count captures its
        # graph: both happen before the timed call
        pkg.lbm_batch_step(b, steps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.lbm_batch_step(b, steps)
        torch.cuda.synchronize()
        bt = time.perf_counter() - t0
        info = pkg.lbm_batch_info(b)
        st = pkg.lbm_batch_wait(b)
        alg = sum(ALG_BYTES[(c.lattice, c.storage)] * c.cells for c in cases)
        peak, _ = measured_peaks()
        out[f"batched_{storage}"] = {"mlups": round(total * steps / bt / 1e6, 1),
                                     "instances": len(cases), "cells": total,
                                     "alg_bytes_per_cell": round(alg / total, 1),
                                     "frac_of_hbm": round(alg * steps / bt / 1e9 / peak, 4),
                                     "mode": "multi-instance launches" if info["mode"] == 1
                                             else "persistent kernel",
                                     "use_graph": info["use_graph"], "threads": info["threads"],
                                     "tile": info["tile"], "items_per_step": info["items_per_step"],
                                     "status": int(st)}
        # the other mode on the same instances, for comparison: the persistent
        # ticketed kernel replayed from its captured graph, or the per-step launches
        other = 0 if info["mode"] == 1 else 1
        pkg.lbm_batch_set_mode(b, other)
        pkg.lbm_batch_step(b, steps)          # captures the graph of the new mode
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.lbm_batch_step(b, steps)
        torch.cuda.synchronize()
        ot = time.perf_counter() - t0
        oinfo = pkg.lbm_batch_info(b)
        ost = pkg.lbm_batch_wait(b)
        key = "persistent" if other == 0 else "multi_launch"
        out[f"batched_{storage}_{key}"] = {
            "mlups": round(total * steps / ot / 1e6, 1),
            "frac_of_hbm": round(alg * steps / ot / 1e9 / peak, 4),
            "mode": "persistent kernel" if other == 0 else "multi-instance launches",
            "use_graph": oinfo["use_graph"], "threads": oinfo["threads"], "tile": oinfo["tile"],
            "status": int(ost)}
    finally:
        pkg.lbm_batch_destroy(b)
        for s in solvers:
            s.close()
    return out


def cpu_sample_case(nx: int = 64):
    """Bounded sample of the workload for the CPU oracle: the same channel
    physics on an nx x 128 x 8 crop (full wall-to-wall height)."""
    wk = dict(WORKLOAD)
    wk.update(nx=nx, nz=8)
    return C.channel_3d(**wk, storage="fp64")


_CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import lbm_cases as C
from oracle import Oracle
import bench
case = bench.cpu_sample_case()
o = Oracle(case, *C.initial_fields(case))
o.step()
n, t0 = 0, time.perf_counter()
while time.perf_counter() - t0 < {seconds}:
    o.step(); n += 1
dt = time.perf_counter() - t0
print(json.dumps(dict(steps=n, seconds=dt, cells=case.cells)))
"""


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def _oracle_workers(code: str, n: int):
    """Run n single-threaded copies of an oracle snippet at once (one per host
    core, fresh interpreters) and return their JSON results."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env) for _ in range(n)]
    out = []
    for pr in procs:
        so, se = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(se[-300:])
        out.append(json.loads(so.strip().splitlines()[-1]))
    return out


def cpu_baseline(seconds: float):
    """The oracle on the host cores: one copy per core on its own crop, all at
    once (weak scaling; cells x steps summed, divided by the longest run), then
    one copy alone for the single-core figure."""
    code = _CPU_SNIPPET.format(root=ROOT, seconds=seconds)
    n = host_cores()
    try:
        allc = _oracle_workers(code, n)
        one = _oracle_workers(code, 1)[0]
    except Exception as exc:
        return {"value": None, "unit": "MLUPS", "cores": n, "kind": "oracle", "error": str(exc)}
    value = sum(d["cells"] * d["steps"] for d in allc) / max(d["seconds"] for d in allc) / 1e6
    single = one["cells"] * one["steps"] / one["seconds"] / 1e6
    return {"value": round(value, 4), "unit": "MLUPS", "cores": n, "kind": "oracle",
            "single_core": round(single, 4),
            "sample": f"FP64 numpy oracle, same channel physics on a 64x128x8 crop per core, "
                      f"{n} single-threaded copies for ~{seconds:.0f} s "
                      f"({sum(d['steps'] for d in allc)} crop steps); single core alone "
                      f"{one['steps']} steps in {one['seconds']:.1f} s"}


_REF_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import lbm_cases as C
from oracle import Oracle
import bench
case = bench.cpu_sample_case({nx})
o = Oracle(case, *C.initial_fields(case))
for _ in range({warmup}):
    o.step()
t0 = time.perf_counter()
for _ in range({steps}):
    o.step()
dt = time.perf_counter() - t0
print(json.dumps(dict(steps={steps}, seconds=dt, cells=case.cells)))
"""


def run_reference(args):
    """The FP64 oracle as it stands on the host cores: one single-threaded copy
    per core, each running --warmup untimed and --steps timed steps (times
    --ref-steps-per-step) on its own crop of the workload; value = cells x steps
    summed over the copies / the longest timed run."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # crop sized so that the whole run stays within a few minutes
    nx = max(4, min(64, int(64 * 200 / max(args.steps, 1)) // 4 * 4))
    per_step = max(1, int(args.ref_steps_per_step))
    n = host_cores()
    code = _REF_SNIPPET.format(root=ROOT, nx=nx, warmup=max(args.warmup, 0),
                               steps=args.steps * per_step)
    res = _oracle_workers(code, n)
    dt = max(d["seconds"] for d in res)
    value = sum(d["cells"] * d["steps"] for d in res) / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "channel_3d_D3Q19_256x128x128_fp32_Re5200_slip_bounce_back_yu",
                       "sample": f"{nx}x128x8 crop of the workload per host core, FP64 oracle"},
            "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": n,
                             "kind": "oracle",
                             "sample": f"{n} single-threaded oracle copies, each on a {nx}x128x8 "
                                       f"crop, {per_step} oracle step(s) per timed step"},
            "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """Short run of one channel case for profilers: set-up, --warmup steps, then
    --steps steps, each launched individually (no graph)."""
    import torch
    import paper_2506_03905_gb300 as pkg
    if args.plate:
        case = C.flat_plate_3d(scheme=args.scheme, storage=args.storage)
    else:
        case = C.channel_3d(re_tau=5200.0, scheme=args.scheme, nx=args.nx, ny=args.ny, nz=args.nz,
                            storage=args.storage)
    s = pkg.Solver(case)
    s.set_fields(*C.initial_fields(case))
    s.step_timed(args.warmup)
    bulk, wall = s.step_timed(args.steps)
    torch.cuda.synchronize()
    s.close()
    print(json.dumps({"profile_case": case.name, "storage": args.storage, "steps": args.steps,
                      "bulk_ms": bulk / args.steps, "wall_ms": wall / args.steps}))


def run_profile_batch(args):
    """Short run of the 96-instance batched sweep for profilers: set-up and
    autotuning, one warm-up launch of 3 steps, then one launch of --steps
    steps."""
    import torch
    import paper_2506_03905_gb300 as pkg
    cases = C.batched_sweep(96, storage=args.storage)
    solvers = []
    for c in cases:
        s = pkg.Solver(c)
        s.set_fields(*C.initial_fields(c))
        solvers.append(s)
    b = pkg.lbm_batch_create([s.ctx for s in solvers])
    try:
        pkg.lbm_batch_step(b, 3)
        torch.cuda.synchronize()
        pkg.lbm_batch_step(b, args.steps)
        torch.cuda.synchronize()
    finally:
        pkg.lbm_batch_destroy(b)
        for s in solvers:
            s.close()
    print(json.dumps({"profile_batch": len(cases), "cells": sum(c.cells for c in cases),
                      "storage": args.storage, "steps": args.steps}))


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-steps-per-step", type=int, default=1)
    ap.add_argument("--profile-batch", action="store_true",
                    help="short run of the 96-instance batched sweep (for ncu)")
    ap.add_argument("--profile-case", action="store_true",
                    help="short per-launch run of one channel case (for ncu)")
    ap.add_argument("--nx", type=int, default=256)
    ap.add_argument("--ny", type=int, default=128)
    ap.add_argument("--nz", type=int, default=64)
    ap.add_argument("--scheme", default="wall_bb")
    ap.add_argument("--plate", action="store_true",
                    help="--profile-case on the 2048x512x8 flat plate instead of the channel")
    ap.add_argument("--storage", default="fp32")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.profile_batch:
        run_profile_batch(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
