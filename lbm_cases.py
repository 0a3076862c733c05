"""Seeded synthetic workloads for the LBM-RANS wall-function solver.

This module only *describes* inputs: lattice sizes, physical parameters,
boundary-condition choices and seeded initial fields in physical units.  It
holds none of the lattice Boltzmann or Spalart-Allmaras arithmetic; both the
FP64 oracle and the CUDA library convert these physical inputs to lattice
units on their own.

The shapes follow the paper's two test cases:

* turbulent channel, Section 4.1.1: half-width h = 1 m, rho0 = 1 kg/m^3,
  nu = 1.5e-5 m^2/s, constant body force g = u_tau^2 / h, initial bulk velocity
  from Dean's correlation Re_b = (8/0.073)^(4/7) Re_tau^(8/7), acoustic time step
  with Mach 0.1 (Table 2 lists the resulting numbers);
* zero-pressure-gradient flat plate, Section 4.2.1: U = 75 m/s, Mach 0.1,
  nu = 1.5e-5 m^2/s (Re = 5e6 per metre), plate leading edge at x = 0, inlet at
  x = -0.2 m, meshes with Delta = 2e-3 / 1e-3 / 5e-4 m (Table 4), free-stream
  nu_tilde / nu = 3.

The channel DNS data and the flat-plate CFL3D reference data the paper compares
against are not available; these synthetic inputs stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

FACES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")
BC_KINDS = ("periodic", "wall_bb", "wall_hrfd", "symmetry", "inlet_zouhe",
            "outlet_zerograd", "freestream", "wall_cai_degrigny")
# bounce-back variants for a wall that is not half-way between lattice nodes:
# none (half-way, Eq. 31), Bouzidi (Eq. 36), Yu (Eq. 37)
BB_INTERP = ("none", "bouzidi", "yu")

NU_AIR = 1.5e-5          # m^2/s, Section 4.1.1 and Section 4.2.1
RHO0 = 1.0               # kg/m^3, Section 4.1.1
MACH = 0.1               # Section 4.2.1 (acoustic scaling, Section 4.1.1)
BETA_STAR = 0.28         # calibrated HRFD blend, Section 4.1.2.1
PLATE_U_INF = 75.0       # m/s, Section 4.2.1


@dataclass
class BC:
    """Boundary condition of one domain face (all quantities physical)."""
    kind: str = "periodic"
    beta: float = BETA_STAR          # HRFD blend of Eq. 27
    ref_node: int = 2                # 1 = B (first node), 2 = F (second node)
    x_start: float = -math.inf       # wall active where cell-centre x >= x_start
    u_in: Tuple[float, float, float] = (0.0, 0.0, 0.0)   # inlet / free-stream velocity
    nut_ratio_in: float = 3.0        # inlet / free-stream nu_tilde / nu
    d_w: float = 0.5                 # wall-to-boundary-node distance / Delta (Section 4.1.2.5)
    interp: str = "none"             # bounce-back walls: "none" | "bouzidi" | "yu"

    def __post_init__(self):
        if self.kind not in BC_KINDS:
            raise ValueError(f"unknown boundary kind {self.kind!r}")
        if self.interp not in BB_INTERP:
            raise ValueError(f"unknown bounce-back interpolation {self.interp!r}")


@dataclass
class Case:
    """One lattice problem.  Units: SI; sizes in cells."""
    name: str
    lattice: str                      # "D2Q9" | "D3Q19"
    nx: int
    ny: int
    nz: int
    dx: float                         # m
    nu: float = NU_AIR                # m^2/s
    rho0: float = RHO0                # kg/m^3
    u_ref: float = 1.0                # m/s, sets the acoustic time step
    mach: float = MACH
    force: Tuple[float, float, float] = (0.0, 0.0, 0.0)   # body acceleration g, m/s^2
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)  # physical coords of the low corner
    collision: str = "bgk"            # "bgk" | "regularized"
    storage: str = "fp32"             # "fp64" | "fp32" | "fp16" | "bf16"
    turbulence: str = "sa"            # "sa" | "laminar"
    wall_law: str = "sa_analytic"     # "sa_analytic" (Eq. 16) | "log"
    kappa: float = 0.41
    B: float = 5.2
    bcs: Dict[str, BC] = field(default_factory=dict)
    u_init: Tuple[float, float, float] = (0.0, 0.0, 0.0)  # m/s
    perturb: float = 0.0              # relative amplitude of the seeded u_x perturbation
    seed: int = 0
    nut_ratio_init: float = 3.0       # initial nu_tilde / nu (floor of the log-layer profile)
    nut_utau: float = 0.0             # m/s; > 0: initial nu_tilde = max(ratio nu, kappa u_tau d)
    steps: int = 100
    u_shift: Optional[float] = None   # storage reference velocity (None: u_init x)

    def __post_init__(self):
        if self.lattice not in ("D2Q9", "D3Q19"):
            raise ValueError(self.lattice)
        if self.lattice == "D2Q9" and self.nz != 1:
            raise ValueError("D2Q9 cases have nz == 1")
        for f in FACES:
            self.bcs.setdefault(f, BC("periodic"))

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Case":
        """Copy with fields replaced; ``bcs`` entries given here override single faces."""
        new_bcs = dict(kw.pop("bcs", {}))
        c = dataclasses.replace(self, **kw)
        c.bcs = {k: dataclasses.replace(v) for k, v in self.bcs.items()}
        c.bcs.update(new_bcs)
        return c


def initial_fields(case: Case):
    """Seeded initial density, velocity and SA working variable (physical units).

    u_x = u_init_x * (1 + perturb * r) with r uniform in [-1, 1) drawn from
    numpy's PCG64 generator seeded with ``case.seed``; u_y, u_z = u_init_y, u_init_z;
    rho = rho0; nu_tilde = nut_ratio_init * nu.  Arrays are indexed [z, y, x]
    (velocity [component, z, y, x]), float64.
    """
    shape = (case.nz, case.ny, case.nx)
    rho = np.full(shape, case.rho0, dtype=np.float64)
    u = np.empty((3,) + shape, dtype=np.float64)
    u[0] = case.u_init[0]
    u[1] = case.u_init[1]
    u[2] = case.u_init[2]
    if case.perturb != 0.0:
        rng = np.random.default_rng(case.seed)
        r = rng.uniform(-1.0, 1.0, size=shape)
        u[0] = case.u_init[0] * (1.0 + case.perturb * r)
    nut = np.full(shape, case.nut_ratio_init * case.nu, dtype=np.float64)
    if case.nut_utau > 0.0:
        # log-layer start: nu_tilde = kappa u_tau d with d the distance to the
        # nearest wall face (boundary nodes d_w Delta from their wall)
        j = np.arange(case.ny, dtype=np.float64)
        d = np.full(case.ny, np.inf)
        for f, dist in (("ymin", j), ("ymax", case.ny - 1 - j)):
            b = case.bcs[f]
            if b.kind in ("wall_bb", "wall_hrfd", "wall_cai_degrigny"):
                d = np.minimum(d, (dist + b.d_w) * case.dx)
        if np.isfinite(d).all():
            prof = np.maximum(case.nut_ratio_init * case.nu, case.kappa * case.nut_utau * d)
            nut[:] = prof[None, :, None]
    return rho, u, nut


# ----------------------------------------------------------------------------
# Channel flow, Section 4.1.1
# ----------------------------------------------------------------------------

def dean_bulk_reynolds(re_tau: float) -> float:
    """Dean's correlation Re_b = (8/0.073)^(4/7) Re_tau^(8/7) (Section 4.1.1)."""
    return (8.0 / 0.073) ** (4.0 / 7.0) * re_tau ** (8.0 / 7.0)


def dean_cfb(re_b: float) -> float:
    """Dean's correlation in friction-coefficient form, C_fb = 0.073 Re_b^(-1/4): with
    C_fb = 2 (u_tau / U_b)^2 = 8 (Re_tau / Re_b)^2 it is the Re_b(Re_tau) relation of
    Section 4.1.1."""
    return 0.073 * re_b ** -0.25


def channel_parameters(re_tau: float, h: float = 1.0, nu: float = NU_AIR):
    """u_tau, g, Re_b, U_b, C_fb, y(y+=50) of Table 2 for a given Re_tau."""
    u_tau = re_tau * nu / h
    g = u_tau ** 2 / h
    re_b = dean_bulk_reynolds(re_tau)
    u_b = re_b * nu / (2.0 * h)
    cfb = 2.0 * (u_tau / u_b) ** 2
    y50 = 50.0 * nu / u_tau
    return dict(u_tau=u_tau, g=g, re_b=re_b, u_b=u_b, cfb=cfb, y_first=y50)


def half_channel_2d(re_tau: float = 2000.0, ny: int = 48, nx: int = 4,
                    storage: str = "fp64", steps: int = 20000) -> Case:
    """2-D D2Q9 half channel: wall at y = 0, symmetry at the centreline y = h.

    Periodic in x; BGK; SA; slip-velocity bounce-back whose wall function is the
    log law (kappa = 0.41, B = 5.2) enforced at the first node; u = 0 initially.
    """
    h = 1.0
    p = channel_parameters(re_tau, h)
    return Case(
        name=f"half_channel_2d_Re{int(re_tau)}_{nx}x{ny}", lattice="D2Q9",
        nx=nx, ny=ny, nz=1, dx=h / ny, u_ref=p["u_b"], force=(p["g"], 0.0, 0.0),
        collision="bgk", storage=storage, turbulence="sa", wall_law="log",
        bcs={"ymin": BC("wall_bb", ref_node=1), "ymax": BC("symmetry")},
        u_init=(0.0, 0.0, 0.0), nut_ratio_init=3.0, steps=steps)


def channel_reynolds_sweep(re_tau: float, scheme: str = "wall_hrfd", n: int = 20,
                           storage: str = "fp64") -> Case:
    """2-D half channel of the Reynolds-number study (Section 4.1.2.6): D2Q9, N = 20
    cells from the wall to the symmetric centreline, periodic in x (4 cells),
    SA model with the SA-consistent wall function (Eq. 16) and the reference
    node F, BGK, initial u = U_b from Dean's correlation, nu_tilde = 3 nu."""
    c = half_channel_2d(re_tau=re_tau, ny=n, nx=4, storage=storage)
    p = channel_parameters(re_tau)
    return c.replace(name=f"channel_re_sweep_Re{int(re_tau)}_{scheme}_N{n}", wall_law="sa_analytic",
                     bcs={"ymin": BC(scheme, ref_node=2)}, u_init=(p["u_b"], 0.0, 0.0))


def channel_3d(re_tau: float = 5200.0, scheme: str = "wall_bb", nx: int = 256,
               ny: int = 128, nz: int = 128, seed: int = 0, storage: str = "fp32",
               collision: str = "bgk", wall_law: str = "sa_analytic",
               ref_node: int = 2, steps: int = 1000, d_w: float = 0.5,
               interp: str = "none", nut_init: str = "log_layer") -> Case:
    """3-D D3Q19 full channel: walls at y = 0 and y = 2h, periodic in x and z.

    The boundary nodes lie d_w Delta from the walls (Section 4.1.2.5; d_w = 1/2
    is the half-way placement), so 2h = (ny - 1 + 2 d_w) Delta; initial
    u_x = U_b (1 +/- 1 %) seeded.  Initial nu_tilde: "log_layer" (default)
    max(3 nu, kappa u_tau d), the log-layer solution of the SA model with d the
    wall distance, or "uniform" 3 nu.  (With the uniform start the BGK channel
    at Re_tau = 5200 on 128 cells begins almost inviscid, tau - 1/2 ~ 1e-4, and
    diverges within ~2000 steps.)
    """
    h = 1.0
    p = channel_parameters(re_tau, h)
    wall = BC(scheme, ref_node=ref_node, d_w=d_w, interp=interp)
    tag = "" if (d_w == 0.5 and interp == "none") else f"_{interp}_dw{d_w:g}"
    return Case(
        name=f"channel_3d_Re{int(re_tau)}_{scheme}{tag}_{nx}x{ny}x{nz}", lattice="D3Q19",
        nx=nx, ny=ny, nz=nz, dx=2.0 * h / (ny - 1 + 2.0 * d_w), u_ref=p["u_b"],
        force=(p["g"], 0.0, 0.0),
        collision=collision, storage=storage, turbulence="sa", wall_law=wall_law,
        bcs={"ymin": wall, "ymax": dataclasses.replace(wall)},
        u_init=(p["u_b"], 0.0, 0.0), perturb=0.01, seed=seed, nut_ratio_init=3.0,
        nut_utau=p["u_tau"] if nut_init == "log_layer" else 0.0, steps=steps)


# ----------------------------------------------------------------------------
# Zero-pressure-gradient flat plate, Section 4.2.1
# ----------------------------------------------------------------------------

def flat_plate_3d(nx: int = 2048, ny: int = 512, nz: int = 8, dx: float = 1e-3,
                  scheme: str = "wall_bb", storage: str = "fp32",
                  collision: str = "regularized", top: str = "freestream",
                  x_inlet: float = -0.2, steps: int = 1000,
                  u_inf: float = PLATE_U_INF, interp: Optional[str] = None) -> Case:
    """3-D D3Q19 flat plate: Zou-He inlet, zero-gradient outlet, free-stream top,
    bottom symmetry for x < 0 and wall for x >= 0, spanwise periodic.
    Initial state: uniform U_inf with nu_tilde / nu = 3.  A bounce-back wall
    uses Yu's rule (Eq. 37) by default, as the paper does on the plate
    (Section 3.2); interp="none" selects half-way bounce-back."""
    if interp is None:
        interp = "yu" if scheme == "wall_bb" else "none"
    bcs = {
        "xmin": BC("inlet_zouhe", u_in=(u_inf, 0.0, 0.0), nut_ratio_in=3.0),
        "xmax": BC("outlet_zerograd"),
        "ymin": BC(scheme, ref_node=2, x_start=0.0, interp=interp),
        "ymax": BC(top, u_in=(u_inf, 0.0, 0.0), nut_ratio_in=3.0),
    }
    return Case(
        name=f"flat_plate_3d_{scheme}_{nx}x{ny}x{nz}", lattice="D3Q19",
        nx=nx, ny=ny, nz=nz, dx=dx, u_ref=u_inf, force=(0.0, 0.0, 0.0),
        origin=(x_inlet, 0.0, 0.0), collision=collision, storage=storage,
        turbulence="sa", wall_law="sa_analytic", bcs=bcs,
        u_init=(u_inf, 0.0, 0.0), nut_ratio_init=3.0, steps=steps)


def flat_plate_2d(nx: int = 1100, ny: int = 250, dx: float = 2e-3,
                  scheme: str = "wall_bb", storage: str = "fp32",
                  collision: str = "regularized", top: str = "symmetry",
                  steps: int = 1000) -> Case:
    """D2Q9 flat plate on the paper's coarse mesh (Table 4: 1100 x 250)."""
    c = flat_plate_3d(nx=nx, ny=ny, nz=1, dx=dx, scheme=scheme, storage=storage,
                      collision=collision, top=top, steps=steps)
    return c.replace(name=f"flat_plate_2d_{scheme}_{nx}x{ny}", lattice="D2Q9")


# ----------------------------------------------------------------------------
# Batched mesh-sensitivity sweep
# ----------------------------------------------------------------------------

def batched_sweep(n: int = 96, seed: int = 2506, storage: str = "fp32",
                  plate_nx_cap: Optional[int] = None) -> List[Case]:
    """Heterogeneous instances for a mesh-sensitivity sweep.

    Instance k: D2Q9 if k is even else D3Q19 (nz = 4); channel if k % 3 != 2
    else flat plate; ny drawn from {16, ..., 256}; channel nx from {4, ..., 64}
    (D2Q9 channels use nx = 4), plate nx = min(4 ny, 1024); channel Re_tau
    log-uniform in [500, 2e4], plate Re per metre log-uniform in [1e6, 1e7];
    slip-velocity bounce-back if k % 4 < 2 else HRFD.  ``plate_nx_cap`` caps the
    plates' nx (same domain, coarser Delta) for parity runs of the same sweep.
    """
    rng = np.random.default_rng(seed)
    ny_choices = [16, 24, 32, 48, 64, 96, 128, 192, 256]
    nx_choices = [4, 8, 16, 32, 64]
    out = []
    for k in range(n):
        lattice = "D2Q9" if k % 2 == 0 else "D3Q19"
        nz = 1 if lattice == "D2Q9" else 4
        plate = (k % 3 == 2)
        scheme = "wall_bb" if k % 4 < 2 else "wall_hrfd"
        ny = int(rng.choice(ny_choices))
        if plate:
            re_m = float(np.exp(rng.uniform(np.log(1e6), np.log(1e7))))
            nx = min(4 * ny, 1024, plate_nx_cap or 1024)
            u_inf = re_m * NU_AIR          # Re per metre = U / nu
            length = 2.048                 # domain length in metres
            dx = length / nx
            c = flat_plate_3d(nx=nx, ny=ny, nz=nz, dx=dx, scheme=scheme,
                              storage=storage, u_inf=u_inf,
                              x_inlet=-0.1 * length)
            c = c.replace(name=f"sweep{k:02d}_plate_{lattice}_{nx}x{ny}x{nz}",
                          lattice=lattice)
        else:
            re_tau = float(np.exp(rng.uniform(np.log(500.0), np.log(2e4))))
            nx = 4 if lattice == "D2Q9" else int(rng.choice(nx_choices))
            c = channel_3d(re_tau=re_tau, scheme=scheme, nx=nx, ny=ny, nz=nz,
                           seed=k, storage=storage)
            c = c.replace(name=f"sweep{k:02d}_channel_{lattice}_{nx}x{ny}x{nz}",
                          lattice=lattice)
        out.append(c)
    return out


def shard_instances(cells: List[int], world: int, rank: int) -> List[int]:
    """Indices of the instances rank `rank` of `world` advances in a sharded sweep.

    Instances are independent, so a sweep shards with no exchange between ranks:
    greedy longest-first assignment of instances to the rank with the fewest
    cells so far (ties to the lower rank), which keeps the per-rank cell counts
    within one instance of each other.
    """
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    load = [0] * world
    owner = [0] * len(cells)
    for i in sorted(range(len(cells)), key=lambda k: (-cells[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += cells[i]
    return [i for i in range(len(cells)) if owner[i] == rank]
