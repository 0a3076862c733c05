"""Long oracle runs whose results the GPU tests read back from tests/golden/oracle/.

The FP64 oracle needs minutes to hours of CPU time for these cases (full-size
lattices, thousands of steps), so ``tests/golden/make_oracle_fixtures.py`` runs
it once, through ``oracle/`` and ``lbm_cases`` only, and stores what the tests
compare: the wall arrays (u_tau per wall node; C_f follows from it), the
velocity of the rows next to each wall, and a seeded sample of cells of the
velocity and eddy-viscosity fields with the fields' maxima (the denominators of
the relative errors).  Nothing here comes from the CUDA path.

Every fixture records the case it was made from; ``load`` refuses a fixture
whose case no longer matches the definition below.
"""
from __future__ import annotations

import dataclasses
import json
import os

import numpy as np

import lbm_cases as C

HERE = os.path.dirname(os.path.abspath(__file__))
FIXDIR = os.path.join(HERE, "golden", "oracle")
SAMPLE = 4096            # cells sampled from each 3-D field
SAMPLE_SEED = 2506


def _channel_full(interp):
    # the benchmark's channel: D3Q19 256 x 128 x 128, Re_tau = 5200, FP32
    scheme = "wall_hrfd" if interp == "hrfd" else "wall_bb"
    return C.channel_3d(re_tau=5200.0, scheme=scheme, d_w=0.5,
                        interp="none" if interp == "hrfd" else interp)


def _plate_window():
    # the 2048 x 512 x 8 plate's physics (Delta = 1e-3 m, inlet at x = -0.2 m,
    # leading edge at x = 0) on its first 256 x 128 x 8 cells
    return C.flat_plate_3d(nx=256, ny=128, nz=8, dx=1e-3, scheme="wall_bb")


def _plate_precision(scheme):
    return C.flat_plate_3d(nx=512, ny=128, nz=4, dx=4e-3, scheme=scheme, collision="regularized")


def _channel_fp16_crop():
    # the benchmark's FP16 channel physics on a 64 x 128 x 8 crop
    return C.channel_3d(re_tau=5200.0, scheme="wall_bb", nx=64, ny=128, nz=8, seed=0, d_w=0.5,
                        interp="yu")


# name -> (case factory, steps)
CASES = {
    "channel_full_halfway_50": (lambda: _channel_full("none"), 50),
    "channel_full_yu_50": (lambda: _channel_full("yu"), 50),
    "channel_full_hrfd_50": (lambda: _channel_full("hrfd"), 50),
    "plate_window_256x128x8_bb_200": (_plate_window, 200),
    "plate_512x128x4_bb_2000": (lambda: _plate_precision("wall_bb"), 2000),
    "plate_512x128x4_hrfd_2000": (lambda: _plate_precision("wall_hrfd"), 2000),
    "channel_crop_64x128x8_yu_2000": (_channel_fp16_crop, 2000),
}


# Reynolds-number study of Section 4.1.2.6 (Fig. 12): converged runs, stopped by
# the criterion of Section 4.1.1 applied per chunk of CFB_CHECK steps
CFB_RE_TAU = (2000.0, 4200.0, 8000.0, 20000.0)
CFB_SCHEMES = ("wall_hrfd", "wall_bb", "wall_cai_degrigny")
CFB_TOL, CFB_CHECK, CFB_MAX = 1e-4, 1000, 200000
CFB_CASES = {f"cfb_Re{int(r)}_{s}": (r, s) for r in CFB_RE_TAU for s in CFB_SCHEMES}


def cfb_case(name):
    r, s = CFB_CASES[name]
    return C.channel_reynolds_sweep(r, s)


def case_signature(case) -> str:
    """Every parameter of the case except its storage type (the oracle is FP64)."""
    d = dataclasses.asdict(case)
    d.pop("storage", None)
    return json.dumps(d, sort_keys=True, default=str)


def _pick(n, k, seed):
    rng = np.random.default_rng(seed)
    return np.arange(n) if n <= k else np.sort(rng.choice(n, size=k, replace=False))


def sample_cells(case):
    """Seeded flat indices (into nz*ny*nx) of the sampled cells: SAMPLE cells of the
    whole lattice, then up to 2 SAMPLE cells of the three rows next to each y face."""
    idx = _pick(case.cells, SAMPLE, SAMPLE_SEED)
    rows = np.array(sorted({0, 1, 2, case.ny - 3, case.ny - 2, case.ny - 1}))
    z, r, x = np.meshgrid(np.arange(case.nz), rows, np.arange(case.nx), indexing="ij")
    near = ((z * case.ny + r) * case.nx + x).ravel()
    near = np.sort(near[_pick(near.size, 2 * SAMPLE, SAMPLE_SEED + 1)])
    return idx, near


def sample_nodes(case):
    """Seeded indices (into nz*nx) of the sampled wall nodes of a face."""
    return _pick(case.nx * case.nz, 2 * SAMPLE, SAMPLE_SEED + 2)


def wall_faces(case):
    return [f for f in ("ymin", "ymax")
            if case.bcs[f].kind in ("wall_bb", "wall_hrfd", "wall_cai_degrigny")]


def reduce_fields(case, fields):
    """What a fixture stores, from a dict of physical fields (oracle or GPU)."""
    idx, near = sample_cells(case)
    u = fields["u"].reshape(3, -1)
    nut = fields["nu_t"].reshape(-1)
    out = {
        "u_sample": u[:, idx], "nut_sample": nut[idx],
        "u_near": u[:, near], "nut_near": nut[near],
        "u_max": np.abs(u).max(axis=1), "nut_max": np.array(np.abs(nut).max()),
    }
    nodes = sample_nodes(case)
    for f in wall_faces(case):
        out["u_tau_" + f] = fields["u_tau_" + f].reshape(-1)[nodes]
        out["u_tau_max_" + f] = np.array(np.abs(fields["u_tau_" + f]).max())
    return out


def path(name):
    return os.path.join(FIXDIR, name + ".npz")


def load_cfb(name):
    """(case, results) of a stored Reynolds-study fixture."""
    case = cfb_case(name)
    p = path(name)
    if not os.path.exists(p):
        raise FileNotFoundError(f"{p} missing: run tests/golden/make_oracle_fixtures.py {name}")
    with np.load(p, allow_pickle=False) as z:
        meta = json.loads(str(z["meta"]))
    if meta["signature"] != case_signature(case):
        raise RuntimeError(f"{p} was made from another case definition: regenerate it")
    return case, meta


def load(name):
    """(case, steps, arrays) of a stored fixture; raises if it is missing or stale."""
    factory, steps = CASES[name]
    case = factory()
    p = path(name)
    if not os.path.exists(p):
        raise FileNotFoundError(f"{p} missing: run tests/golden/make_oracle_fixtures.py {name}")
    with np.load(p, allow_pickle=False) as z:
        arrays = {k: z[k] for k in z.files}
    meta = json.loads(str(arrays.pop("meta")))
    if meta["signature"] != case_signature(case) or meta["steps"] != steps:
        raise RuntimeError(f"{p} was made from another case definition: regenerate it")
    return case, steps, arrays
