"""GB300-native LBM-RANS wall-function solver (Ponsin & Lozano, arXiv 2506.03905).

Thin ctypes binding of the C ABI in ``include/lbm.h``: argument marshalling
only, every step of the method runs in the CUDA library ``liblbm_gb300.so``.
Functions keep the C names (``lbm_create``, ``lbm_set_bc``, ``lbm_set_fields``,
``lbm_step``, ``lbm_fields``, ``lbm_destroy`` ...).  :class:`Solver` wraps one
context with PyTorch's caching allocator and current CUDA stream.

There is no CPU fallback: importing works without a GPU, but every call that
needs the library raises if it cannot be loaded.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Dict, Optional, Sequence

import numpy as np

from . import build as _build

__all__ = [
    "lib", "LbmConfig", "LbmBC", "LbmDiag", "Solver", "LbmError",
    "lbm_create", "lbm_set_bc", "lbm_set_fields", "lbm_step", "lbm_step_timed", "lbm_fields",
    "lbm_diagnostics", "lbm_state_bytes", "lbm_get_state", "lbm_set_state", "lbm_destroy",
    "lbm_last_error", "lbm_lattice_params", "lbm_batch_create", "lbm_batch_step",
    "lbm_batch_tune", "lbm_batch_destroy", "lbm_batch_last_error", "lbm_moments_noalloc",
    "lbm_kernel_launches", "lbm_run_to_convergence", "lbm_batch_wait", "lbm_batch_set_wait_limit",
    "lbm_batch_info", "lbm_steps_done", "lbm_set_wait_limit", "lbm_batch_set_mode",
]

LIB_PATH = _build.LIB

# enums of include/lbm.h
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ENEWTON, \
    LBM_EUNSUPPORTED = range(8)
STATUS_NAMES = ["LBM_OK", "LBM_EINVAL", "LBM_ENOMEM", "LBM_ECUDA", "LBM_ENONFINITE",
                "LBM_ETIMEOUT", "LBM_ENEWTON", "LBM_EUNSUPPORTED"]
LATTICE = {"D2Q9": 9, "D3Q19": 19}
COLLISION = {"bgk": 0, "regularized": 1}
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2, "fp64": 3}
TURBULENCE = {"sa": 0, "laminar": 1}
WALL_LAW = {"sa_analytic": 0, "log": 1}
BC_KIND = {"periodic": 0, "wall_bb": 1, "wall_hrfd": 2, "symmetry": 3, "inlet_zouhe": 4,
           "outlet_zerograd": 5, "freestream": 6, "wall_cai_degrigny": 7}
IBB = {"none": 0, "bouzidi": 1, "yu": 2}
FACES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")
FIELD = {"rho": 1 << 0, "u": 1 << 1, "nu_t": 1 << 2, "nu_tilde": 1 << 3,
         "u_tau_ymin": 1 << 4, "u_tau_ymax": 1 << 5, "cf_ymin": 1 << 6, "cf_ymax": 1 << 7}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class LbmConfig(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("nu", ctypes.c_double), ("rho0", ctypes.c_double),
        ("u_ref", ctypes.c_double), ("mach", ctypes.c_double),
        ("force", ctypes.c_double * 3), ("origin", ctypes.c_double * 3),
        ("collision", ctypes.c_int), ("storage", ctypes.c_int), ("turbulence", ctypes.c_int),
        ("wall_law", ctypes.c_int), ("kappa", ctypes.c_double), ("B", ctypes.c_double),
        ("u_shift", ctypes.c_double), ("staging", ctypes.c_int), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
    ]


class LbmBC(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("beta", ctypes.c_double), ("ref_node", ctypes.c_int),
        ("x_start", ctypes.c_double), ("u_in", ctypes.c_double * 3),
        ("nut_ratio_in", ctypes.c_double), ("d_w", ctypes.c_double), ("interp", ctypes.c_int),
    ]


class LbmDiag(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3),
        ("mean_u_tau", ctypes.c_double * 2), ("max_rel_du_tau", ctypes.c_double),
        ("nonfinite", ctypes.c_int), ("newton_failures", ctypes.c_int),
    ]


class LbmError(RuntimeError):
    def __init__(self, status, where, msg=""):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name} {msg}".strip())
        self.status = status


_lib = None
_P = ctypes.c_void_p


def lib():
    """Load (building first if needed) the CUDA library; raise if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing and could not be built")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "lbm_create": (ctypes.c_int, [ctypes.POINTER(LbmConfig), ctypes.POINTER(_P)]),
        "lbm_set_bc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(LbmBC)]),
        "lbm_set_fields": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
        "lbm_step": (ctypes.c_int, [_P, ctypes.c_int]),
        "lbm_step_timed": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
        "lbm_fields": (ctypes.c_int, [_P, ctypes.c_uint, ctypes.POINTER(_P), ctypes.c_int]),
        "lbm_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(LbmDiag)]),
        "lbm_state_bytes": (ctypes.c_size_t, [_P]),
        "lbm_get_state": (ctypes.c_int, [_P, _P]),
        "lbm_set_state": (ctypes.c_int, [_P, _P]),
        "lbm_destroy": (None, [_P]),
        "lbm_last_error": (ctypes.c_char_p, [_P]),
        "lbm_kernel_launches": (ctypes.c_ulonglong, [_P]),
        "lbm_run_to_convergence": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int,
                                                  ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong),
                                                  ctypes.POINTER(ctypes.c_double)]),
        "lbm_lattice_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
        "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)]),
        "lbm_batch_step": (ctypes.c_int, [_P, ctypes.c_int]),
        "lbm_batch_tune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
        "lbm_batch_destroy": (None, [_P]),
        "lbm_batch_last_error": (ctypes.c_char_p, [_P]),
        "lbm_moments_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
        "lbm_steps_done": (ctypes.c_longlong, [_P]),
        "lbm_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_longlong]),
        "lbm_batch_wait": (ctypes.c_int, [_P]),
        "lbm_batch_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_longlong]),
        "lbm_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
        "lbm_batch_set_mode": (ctypes.c_int, [_P, ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status, where, ctx=None):
    if status != LBM_OK:
        msg = lbm_last_error(ctx)
        raise LbmError(status, where, msg)


# ----------------------------------------------------------------- raw calls
def lbm_create(cfg: LbmConfig):
    h = _P()
    st = lib().lbm_create(ctypes.byref(cfg), ctypes.byref(h))
    _check(st, "lbm_create")
    return h


def lbm_set_bc(ctx, face: int, bc: LbmBC):
    _check(lib().lbm_set_bc(ctx, face, ctypes.byref(bc)), "lbm_set_bc", ctx)


def lbm_set_fields(ctx, rho_ptr, u_ptr, nt_ptr, on_device: bool):
    _check(lib().lbm_set_fields(ctx, rho_ptr, u_ptr, nt_ptr, int(on_device)), "lbm_set_fields", ctx)


def lbm_step(ctx, nsteps: int):
    _check(lib().lbm_step(ctx, int(nsteps)), "lbm_step", ctx)


def lbm_step_timed(ctx, nsteps: int):
    """(bulk rows, wall pre-pass, inner rows) kernel milliseconds over nsteps."""
    ms = (ctypes.c_float * 3)()
    _check(lib().lbm_step_timed(ctx, int(nsteps), ms), "lbm_step_timed", ctx)
    return float(ms[0]), float(ms[1]), float(ms[2])


def lbm_fields(ctx, mask: int, ptrs: Sequence[int], on_device: bool):
    arr = (_P * max(1, len(ptrs)))(*ptrs)
    return lib().lbm_fields(ctx, ctypes.c_uint(mask), arr, int(on_device))


def lbm_diagnostics(ctx) -> LbmDiag:
    d = LbmDiag()
    _check(lib().lbm_diagnostics(ctx, ctypes.byref(d)), "lbm_diagnostics", ctx)
    return d


def lbm_state_bytes(ctx) -> int:
    return int(lib().lbm_state_bytes(ctx))


def lbm_get_state(ctx) -> np.ndarray:
    buf = np.empty(lbm_state_bytes(ctx), dtype=np.uint8)
    _check(lib().lbm_get_state(ctx, buf.ctypes.data), "lbm_get_state", ctx)
    return buf


def lbm_set_state(ctx, buf: np.ndarray):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    if buf.size != lbm_state_bytes(ctx):
        raise ValueError("state buffer has the wrong size")
    _check(lib().lbm_set_state(ctx, buf.ctypes.data), "lbm_set_state", ctx)


def lbm_destroy(ctx):
    lib().lbm_destroy(ctx)


def lbm_last_error(ctx=None) -> str:
    s = lib().lbm_last_error(ctx)
    return s.decode() if s else ""


def lbm_run_to_convergence(ctx, tol: float = 1e-4, check_every: int = 1000,
                           max_steps: int = 1_000_000):
    """Returns (steps taken, last relative u_tau change); see include/lbm.h."""
    n = ctypes.c_longlong(0)
    r = ctypes.c_double(0.0)
    _check(lib().lbm_run_to_convergence(ctx, tol, check_every, max_steps, ctypes.byref(n),
                                        ctypes.byref(r)), "lbm_run_to_convergence", ctx)
    return int(n.value), float(r.value)


def lbm_kernel_launches(ctx) -> int:
    return int(lib().lbm_kernel_launches(ctx))


def lbm_lattice_params(ctx):
    out = (ctypes.c_double * 6)()
    _check(lib().lbm_lattice_params(ctx, out), "lbm_lattice_params", ctx)
    return dict(dt=out[0], nu=out[1], tau0=out[2], F=(out[3], out[4], out[5]))


def lbm_batch_create(ctxs):
    arr = (_P * len(ctxs))(*[c.value if isinstance(c, _P) else c for c in ctxs])
    h = _P()
    st = lib().lbm_batch_create(arr, len(ctxs), ctypes.byref(h))
    if st != LBM_OK:
        raise LbmError(st, "lbm_batch_create", lbm_batch_last_error(None))
    return h


def lbm_batch_step(b, nsteps: int):
    st = lib().lbm_batch_step(b, int(nsteps))
    if st != LBM_OK:
        raise LbmError(st, "lbm_batch_step", lbm_batch_last_error(b))


def lbm_batch_tune(b):
    best = (ctypes.c_int * 2)()
    st = lib().lbm_batch_tune(b, best)
    if st != LBM_OK:
        raise LbmError(st, "lbm_batch_tune", lbm_batch_last_error(b))
    return int(best[0]), int(best[1])


def lbm_batch_destroy(b):
    lib().lbm_batch_destroy(b)


def lbm_batch_wait(b) -> int:
    """Raw status: LBM_OK, or LBM_ETIMEOUT if a bounded wait of the last launch gave up."""
    return lib().lbm_batch_wait(b)


def lbm_batch_set_wait_limit(b, polls: int):
    st = lib().lbm_batch_set_wait_limit(b, int(polls))
    if st != LBM_OK:
        raise LbmError(st, "lbm_batch_set_wait_limit", lbm_batch_last_error(b))


def lbm_batch_info(b):
    """dict(threads, tile, use_graph, items_per_step, mode) of a batch."""
    out = (ctypes.c_int * 5)()
    st = lib().lbm_batch_info(b, out)
    if st != LBM_OK:
        raise LbmError(st, "lbm_batch_info", lbm_batch_last_error(b))
    return dict(threads=out[0], tile=out[1], use_graph=bool(out[2]), items_per_step=out[3],
                mode=out[4])


def lbm_batch_set_mode(b, mode: int):
    """0: persistent ticketed kernel, 1: per-step multi-instance launches, -1: autotuned."""
    st = lib().lbm_batch_set_mode(b, int(mode))
    if st != LBM_OK:
        raise LbmError(st, "lbm_batch_set_mode", lbm_batch_last_error(b))


def lbm_steps_done(ctx) -> int:
    return int(lib().lbm_steps_done(ctx))


def lbm_set_wait_limit(ctx, polls: int):
    _check(lib().lbm_set_wait_limit(ctx, int(polls)), "lbm_set_wait_limit", ctx)


def lbm_moments_noalloc(f_ptr, lattice: int, storage: int, nx: int, ny: int, nz: int,
                        pitch: int, out_ptr, stream=0) -> int:
    """Raw status of the allocation-free mass/momentum reduction (see include/lbm.h)."""
    return lib().lbm_moments_noalloc(f_ptr, lattice, storage, nx, ny, nz, pitch, out_ptr, stream)


def lbm_batch_last_error(b=None) -> str:
    s = lib().lbm_batch_last_error(b)
    return s.decode() if s else ""


# ----------------------------------------------------------------- solver
def config_from_case(case, stream=0, staging=0) -> LbmConfig:
    c = LbmConfig()
    c.lattice = LATTICE[case.lattice]
    c.nx, c.ny, c.nz = case.nx, case.ny, case.nz
    c.dx, c.nu, c.rho0, c.u_ref, c.mach = case.dx, case.nu, case.rho0, case.u_ref, case.mach
    c.force = (ctypes.c_double * 3)(*case.force)
    c.origin = (ctypes.c_double * 3)(*case.origin)
    c.collision = COLLISION[case.collision]
    c.storage = STORAGE[case.storage]
    c.turbulence = TURBULENCE[case.turbulence]
    c.wall_law = WALL_LAW[case.wall_law]
    c.kappa, c.B = case.kappa, case.B
    # stored populations are deviations from the equilibrium at the mean flow
    shift = getattr(case, "u_shift", None)
    c.u_shift = case.u_init[0] if shift is None else shift
    c.staging = int(staging)
    c.stream = stream
    return c


def bc_struct(bc) -> LbmBC:
    b = LbmBC()
    b.kind = BC_KIND[bc.kind]
    b.beta = bc.beta
    b.ref_node = bc.ref_node
    b.x_start = bc.x_start if math.isfinite(bc.x_start) else -math.inf
    b.u_in = (ctypes.c_double * 3)(*bc.u_in)
    b.nut_ratio_in = bc.nut_ratio_in
    b.d_w = bc.d_w
    b.interp = IBB[bc.interp]
    return b


class Solver:
    """One lattice on the current CUDA device.

    ``case`` provides the attributes of a case description (lattice, sizes,
    physical parameters, ``bcs`` per face ...).  Device memory comes from
    PyTorch's caching allocator and work is enqueued on PyTorch's current
    stream of the device.
    """

    def __init__(self, case, device: int = 0, use_torch_allocator: bool = True,
                 tma_staging: bool = False):
        import torch
        self.torch = torch
        self.case = case
        self.device = device
        torch.cuda.set_device(device)
        self.stream = torch.cuda.current_stream(device)
        cfg = config_from_case(case, self.stream.cuda_stream, staging=int(tma_staging))
        self._cbs = None
        if use_torch_allocator:
            stream = self.stream

            def _alloc(size, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), device, stream)
                except Exception:  # out of memory: report NULL to the library
                    return None

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cbs = (ALLOC_FN(_alloc), FREE_FN(_free))
            cfg.alloc, cfg.free = self._cbs
        self.cfg = cfg
        self.ctx = lbm_create(cfg)
        for i, face in enumerate(FACES):
            lbm_set_bc(self.ctx, i, bc_struct(case.bcs[face]))
        self.n = case.nx * case.ny * case.nz

    # -- state
    def set_fields(self, rho, u, nut):
        """Initial physical fields (numpy float64 host arrays or CUDA tensors)."""
        torch = self.torch
        if isinstance(rho, torch.Tensor):
            rho, u, nut = (t.contiguous().to(torch.float64) for t in (rho, u, nut))
            self._keep = (rho, u, nut)
            lbm_set_fields(self.ctx, rho.data_ptr(), u.data_ptr(), nut.data_ptr(), True)
        else:
            rho, u, nut = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, u, nut))
            lbm_set_fields(self.ctx, rho.ctypes.data, u.ctypes.data, nut.ctypes.data, False)

    def step(self, n: int = 1):
        lbm_step(self.ctx, n)

    def step_timed(self, n: int):
        """(bulk rows, wall pre-pass) kernel milliseconds over n steps."""
        return lbm_step_timed(self.ctx, n)[:2]

    def step_timed3(self, n: int):
        """(bulk rows, wall pre-pass, inner rows) kernel milliseconds over n steps."""
        return lbm_step_timed(self.ctx, n)

    def fields(self, names: Sequence[str] = ("rho", "u", "nu_t", "nu_tilde"),
               device: bool = False, check: bool = True) -> Dict[str, object]:
        """Physical-unit fields as numpy float64 arrays (or CUDA tensors if device)."""
        c = self.case
        shape3 = (c.nz, c.ny, c.nx)
        shapes = {"rho": shape3, "u": (3,) + shape3, "nu_t": shape3, "nu_tilde": shape3,
                  "u_tau_ymin": (c.nz, c.nx), "u_tau_ymax": (c.nz, c.nx),
                  "cf_ymin": (c.nz, c.nx), "cf_ymax": (c.nz, c.nx)}
        order = sorted(names, key=lambda k: FIELD[k])
        mask = 0
        for k in order:
            mask |= FIELD[k]
        out = {}
        if device:
            torch = self.torch
            for k in order:
                out[k] = torch.empty(shapes[k], dtype=torch.float64, device=f"cuda:{self.device}")
            ptrs = [out[k].data_ptr() for k in order]
        else:
            for k in order:
                out[k] = np.empty(shapes[k], dtype=np.float64)
            ptrs = [out[k].ctypes.data for k in order]
        st = lbm_fields(self.ctx, mask, ptrs, device)
        if check:
            _check(st, "lbm_fields", self.ctx)
        self.last_status = st
        return out

    def diagnostics(self) -> LbmDiag:
        return lbm_diagnostics(self.ctx)

    def get_state(self):
        return lbm_get_state(self.ctx)

    def set_state(self, buf):
        lbm_set_state(self.ctx, buf)

    def lattice_params(self):
        return lbm_lattice_params(self.ctx)

    def run_to_convergence(self, tol: float = 1e-4, check_every: int = 1000,
                           max_steps: int = 1_000_000):
        return lbm_run_to_convergence(self.ctx, tol, check_every, max_steps)

    def kernel_launches(self) -> int:
        return lbm_kernel_launches(self.ctx)

    def steps_done(self) -> int:
        return lbm_steps_done(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
