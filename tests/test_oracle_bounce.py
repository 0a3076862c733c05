"""Pins of the bounce-back rules for a wall off the half-way position
(Section 3.2, Eqs. 36-37) and of the wall-distance parameter d_w of
Section 4.1.2.5, against what the mathematics fixes:

* a fluid in equilibrium at the wall velocity is a fixed point of every rule
  at every q (constant data are interpolated exactly; the moving-wall term
  turns f^eq_i into f^eq_opp(i));
* Bouzidi's two branches both reduce to half-way bounce-back (Eq. 31) at
  q = 1/2, for single links and for whole channel runs;
* laminar Poiseuille flow between walls placed d_w off the boundary nodes
  converges at second order to the parabola through the true wall positions
  (a wrong interpolation weight or wall position leaves a first-order error);
* the wall-function geometry with d_w: Eq. 35 with Delta_w = y_B = d_w and
  the regularized u_B = u_tau u+(y_B+).
"""
import math

import numpy as np
import pytest

import lbm_cases as C
from oracle import Oracle, bounce as BB, lattice as L, wallfn as W


def make(case):
    return Oracle(case, *C.initial_fields(case))


QS = [0.1, 0.3, 0.5, 0.64, 0.9, 1.0]


@pytest.mark.parametrize("rule", ["bouzidi", "yu"])
@pytest.mark.parametrize("q", QS)
def test_equilibrium_at_wall_velocity_is_fixed(rule, q):
    vs = L.VelocitySet("D3Q19")
    rho = 1.037
    uw = np.array([0.043, 0.0, -0.021])
    feq = L.equilibrium(vs, np.array(rho), uw)
    for i in np.where(vs.c[:, 1] < 0)[0]:            # links into a ymin wall
        o = vs.opp[i]
        mw = 2.0 * vs.w[i] * rho * (vs.cf[i] @ uw) / L.CS2
        got = BB.RULES[rule](q, feq[i], feq[i], feq[o], mw)
        assert abs(got - feq[o]) < 1e-16


@pytest.mark.parametrize("seed", range(5))
def test_bouzidi_reduces_to_half_way_at_one_half(seed):
    r = np.random.default_rng(seed).uniform(0.0, 0.1, size=4)
    half = BB.halfway(r[0], r[3])
    assert BB.bouzidi(0.5, *r) == pytest.approx(half, abs=1e-17)
    # and the two branches meet there
    lo = BB.bouzidi(0.5 - 1e-9, *r)
    assert abs(lo - half) < 1e-9


@pytest.mark.parametrize("scheme_q", [0.5])
def test_bouzidi_channel_run_equals_half_way(scheme_q):
    base = C.channel_3d(re_tau=2000.0, nx=6, ny=12, nz=3, seed=5)
    a = make(base)
    b = make(C.channel_3d(re_tau=2000.0, nx=6, ny=12, nz=3, seed=5, d_w=scheme_q,
                          interp="bouzidi"))
    a.run(12)
    b.run(12)
    assert np.abs(a.fs - b.fs).max() < 1e-16
    assert np.abs(a.utau["ymin"] - b.utau["ymin"]).max() == 0.0


def poiseuille_error(interp, d_w, ny, tau=0.8, umax=0.01):
    """Relative max error of the steady laminar profile against the parabola
    g/(2 nu) y (H - y) with the walls d_w below the first and above the last
    node: y_j = j + d_w, H = ny - 1 + 2 d_w (lattice units)."""
    bc = C.BC("wall_bb", d_w=d_w, interp=interp)
    c = C.half_channel_2d(ny=ny, nx=1).replace(
        turbulence="laminar", bcs={"ymin": bc, "ymax": C.BC("wall_bb", d_w=d_w, interp=interp)})
    o = make(c)
    o.nu = (tau - 0.5) / 3.0
    H = ny - 1 + 2.0 * d_w
    g = 8.0 * o.nu * umax / H ** 2
    o.F = np.array([g, 0.0, 0.0])
    # twelve e-folds of the slowest diffusive mode
    o.run(int(12 * H * H / (o.nu * math.pi ** 2)) + 100)
    y = np.arange(ny) + d_w
    ua = g / (2.0 * o.nu) * y * (H - y)
    assert np.abs(o.u[1]).max() < 1e-15
    return np.abs(o.u[0, 0, :, 0] - ua).max() / ua.max()


@pytest.mark.parametrize("interp,d_w", [("bouzidi", 0.3), ("bouzidi", 0.7), ("yu", 0.3),
                                        ("yu", 0.8)])
def test_poiseuille_second_order_off_half_way(interp, d_w):
    e8 = poiseuille_error(interp, d_w, 8)
    e16 = poiseuille_error(interp, d_w, 16)
    assert e16 < 1e-2
    assert e8 / e16 > 3.3          # second order (a misplaced wall gives ~2)


def test_bb_prepass_with_wall_distance():
    """Eq. 35 with Delta_w = y_B = d_w and nu_t|_B = nu kappa y_B+:
    u_B - u_w = u_tau y_B+ / (1 + kappa y_B+), y_B+ = u_tau d_w / nu; the
    Newton reference height of node F is 1 + d_w."""
    d_w = 0.3
    c = C.channel_3d(re_tau=2000.0, nx=6, ny=12, nz=1, seed=3, d_w=d_w,
                     interp="yu").replace(lattice="D2Q9")
    o = make(c)
    o.run(3)
    uF_prev = o.u[0, :, 1, :].copy()
    nt_new = o.nt.copy()
    uw, _ = o.bb_prepass("ymin", nt_new)
    ut = o.utau["ymin"]
    ypB = ut * d_w / o.nu
    uB = o.u[0, :, 0, :]
    assert np.allclose(uB - uw[0], ut * ypB / (1 + W.KAPPA * ypB), rtol=1e-12)
    assert np.allclose(nt_new[:, 0, :], o.nu * W.KAPPA * ypB, rtol=1e-14)
    assert np.allclose(ut * W.u_plus_sa(ut * (1.0 + d_w) / o.nu), np.abs(uF_prev), rtol=1e-12)


def test_hrfd_boundary_velocity_with_wall_distance():
    d_w = 0.7
    c = C.channel_3d(re_tau=2000.0, scheme="wall_hrfd", nx=6, ny=12, nz=3, seed=3, d_w=d_w)
    o = make(c)
    o.run(4)
    nt_new = o.sa_update()
    f = o.hrfd(o.x_faces(o.y_faces(o.stream(), {})), nt_new)
    fB = f[:, :, 0, :]
    m1 = np.einsum("ia,i...->a...", o.vs.cf, fB)
    ut = o.utau["ymin"]
    yp = ut * d_w / o.nu
    speed = np.sqrt(m1[0] ** 2 + m1[2] ** 2) / fB.sum(0)
    assert np.allclose(speed, ut * W.u_plus_sa(yp), rtol=1e-13)
    assert np.allclose(nt_new[:, 0, :], o.nu * W.KAPPA * yp, rtol=1e-14)


def test_wall_distance_of_the_sa_model():
    """d = j + d_w from the ymin wall and (ny - 1 - j) + d_w from the ymax wall."""
    d_w = 0.35
    c = C.channel_3d(re_tau=2000.0, nx=4, ny=10, nz=1, d_w=d_w, interp="bouzidi").replace(
        lattice="D2Q9")
    o = make(c)
    j = np.arange(10.0)
    d = np.minimum(j + d_w, 9 - j + d_w)
    assert np.allclose(o.inv_d2[0, :, 0], 1.0 / d ** 2, rtol=1e-15)


def test_invalid_wall_distance_rejected():
    with pytest.raises(ValueError):
        make(C.channel_3d(nx=4, ny=8, nz=1, d_w=0.3).replace(lattice="D2Q9"))   # half-way at 0.3
    with pytest.raises(ValueError):
        make(C.channel_3d(nx=4, ny=8, nz=1, d_w=1.3, interp="yu").replace(lattice="D2Q9"))
