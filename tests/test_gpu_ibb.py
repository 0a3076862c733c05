"""GPU (C ABI) versus the FP64 oracle for walls that are not half-way between
lattice nodes (Section 4.1.2.5): interpolated bounce-back (Bouzidi, Eq. 36;
Yu, Eq. 37) and the regularized walls with the boundary node d_w Delta from
the wall.  Same tolerances as the other parity tests (FP32 1e-5, FP64 1e-9
relative in the max norm)."""
import numpy as np
import pytest

import lbm_cases as C
from test_gpu_parity import TOL, compare, rel, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("interp,d_w", [("bouzidi", 0.3), ("bouzidi", 0.7), ("yu", 0.3),
                                        ("yu", 0.5), ("bouzidi", 1.0)])
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_channel_interpolated_bounce_back(interp, d_w, storage):
    case = C.channel_3d(re_tau=4200.0, nx=40, ny=20, nz=5, seed=6, storage=storage, d_w=d_w,
                        interp=interp)
    compare(case, 120, TOL[storage])


@pytest.mark.parametrize("scheme", ["wall_hrfd", "wall_cai_degrigny"])
@pytest.mark.parametrize("d_w", [0.3, 0.7])
def test_channel_regularized_wall_distance(scheme, d_w):
    case = C.channel_3d(re_tau=4200.0, scheme=scheme, nx=40, ny=20, nz=5, seed=7, d_w=d_w)
    compare(case, 120, TOL["fp32"])


@pytest.mark.parametrize("interp", ["bouzidi", "yu"])
@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_flat_plate_interpolated(interp, lattice):
    """Leading edge, x faces (the F node of a diagonal link leaving the outlet
    column stays in that column), Zou-He inlet, free-stream top."""
    nz = 1 if lattice == "D2Q9" else 3
    case = C.flat_plate_3d(nx=70, ny=22, nz=nz, dx=3e-2).replace(
        lattice=lattice,
        bcs={"ymin": C.BC("wall_bb", ref_node=2, x_start=0.0, d_w=0.35, interp=interp)})
    compare(case, 150, TOL["fp32"])


def test_bouzidi_at_one_half_matches_half_way():
    base = C.channel_3d(re_tau=4200.0, nx=40, ny=20, nz=5, seed=6)
    a = run_gpu(base, 60)
    b = run_gpu(C.channel_3d(re_tau=4200.0, nx=40, ny=20, nz=5, seed=6, d_w=0.5,
                             interp="bouzidi"), 60)
    for k in ("u", "nu_t", "u_tau_ymin", "u_tau_ymax"):
        assert rel(b[k], a[k]) < 1e-6, k


def test_laminar_poiseuille_off_half_way():
    """SA off, Yu walls at d_w = 0.3: the GPU run matches the oracle run at
    steady state, whose error against the parabola through the true walls is
    second order (pinned on the CPU)."""
    case = C.half_channel_2d(ny=16, nx=4, storage="fp64").replace(
        turbulence="laminar",
        bcs={"ymin": C.BC("wall_bb", d_w=0.3, interp="yu"),
             "ymax": C.BC("wall_bb", d_w=0.3, interp="yu")})
    compare(case, 400, TOL["fp64"])


def test_invalid_wall_distance_rejected():
    import paper_2506_03905_gb300 as pkg
    bad = [C.channel_3d(nx=8, ny=8, nz=2, d_w=0.3),                     # half-way at 0.3
           C.channel_3d(nx=8, ny=8, nz=2, d_w=1.5, interp="yu"),
           C.channel_3d(nx=8, ny=8, nz=2, scheme="wall_hrfd").replace(
               bcs={"ymin": C.BC("wall_hrfd", interp="yu")})]
    for case in bad:
        with pytest.raises(pkg.LbmError):
            s = pkg.Solver(case)
            s.close()
