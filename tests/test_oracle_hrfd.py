"""Pins of the oracle's regularized wall nodes (Section 3.1) against closed forms.

The reconstruction of Eq. 19 with Eq. 26 puts a non-equilibrium second moment
of exactly -2 rho_B tau_eff c_s^2 S_ab into the populations of a wall node
(the lattice's fourth-order isotropy turns sum_i w_i c_ia c_ib Q_i:S into
2 c_s^4 S_ab).  The tests below prescribe a previous-step velocity whose
finite differences are known in closed form, post-stream populations whose
moments are known in closed form, and then compare the moments of the rebuilt
populations with the strain rate written out from Eqs. 15, 27-28 (HRFD) and
Eq. 29 (Cai-Degrigny):

* wall-normal derivative: beta u_tau^2/nu du+/dy+(y_B+) t + (1 - beta) times
  the one-sided difference of Eq. 28, which is exact on a quadratic profile
  (u_x = a + b j + c j^2 at row j gives b + 2 c j_B along the inward normal);
* tangential derivatives: central differences of sine waves along x and z,
  (sin(k(x+1)) - sin(k(x-1)))/2 = cos(k x) sin(k);
* u_tau from the tangential speed at F after streaming (Eqs. 20-22) by a
  root finder independent of the oracle's Newton iteration, and
  u_B = u_tau u+(y_B+) along t (Section 3.1);
* rho_B of Eq. 23, which for a post-stream state at an equilibrium without
  wall-normal velocity equals its density exactly;
* tau_eff of Eq. 26 from the previous step's nu_tilde at B.

A planted error in beta, in a coefficient of Eq. 28, in the time level of the
velocities that enter Eq. 28, or in the sign of the inward normal moves the
rebuilt moments away from these values.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import lbm_cases as C
from oracle import Oracle, lattice as L, sa, wallfn as W

NX, NY, NZ = 8, 12, 4


def _setup(scheme, beta, lattice="D3Q19", U_F=0.05, rho_B=1.013, u_Bpar=0.021, nt0=None):
    nz = 1 if lattice == "D2Q9" else NZ
    case = C.channel_3d(re_tau=2000.0, scheme=scheme, nx=NX, ny=NY, nz=nz, seed=1)
    case = case.replace(lattice=lattice, force=(0.0, 0.0, 0.0),
                        bcs={f: C.BC(scheme, beta=beta, ref_node=2) for f in ("ymin", "ymax")})
    o = Oracle(case, *C.initial_fields(case))
    vs = o.vs
    # previous-step velocity: quadratic in the row index for u_x, with sine waves
    # along x (in u_y) and along z (in u_x, 3-D only)
    j = np.arange(NY, dtype=np.float64)[None, :, None]
    x = np.arange(NX, dtype=np.float64)[None, None, :]
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    a, b, c = 0.03, 2.0e-3, -7.0e-5
    e, g = 4.0e-4, (3.0e-4 if nz > 1 else 0.0)
    kx, kz = 2 * math.pi / NX, 2 * math.pi / nz
    u = np.zeros((3, nz, NY, NX))
    u[0] = a + b * j + c * j * j + g * np.sin(kz * z)
    u[1] = e * np.sin(kx * x) + 0.0 * j
    o.u = u
    nt0 = 40.0 * o.nu if nt0 is None else nt0
    o.nt = np.full((nz, NY, NX), nt0)
    # post-stream populations: equilibria with known moments, no wall-normal velocity
    rho = np.ones((nz, NY, NX))
    uu = np.zeros((3, nz, NY, NX))
    uu[0] = 0.04
    for row in (1, NY - 2):                          # reference nodes F
        uu[0][:, row, :] = U_F
    for row in (0, NY - 1):                          # boundary nodes B
        rho[:, row, :] = rho_B
        uu[0][:, row, :] = u_Bpar
    f = L.equilibrium(vs, rho, uu)
    geo = dict(a=a, b=b, c=c, e=e, g=g, kx=kx, kz=kz, nt0=nt0, rho_B=rho_B, U_F=U_F, nz=nz)
    return o, f, geo


def _u_tau(o, U, y):
    """Root of U = u_tau u+(u_tau y / nu) by Brent's method (not the oracle's Newton)."""
    return brentq(lambda ut: ut * W.u_plus_sa(ut * y / o.nu) - U, 1e-12, 10.0 * U, xtol=1e-18,
                  rtol=1e-15, maxiter=400)


def _neq_second_moment(vs, fB):
    rho = fB.sum(0)
    m1 = np.einsum("ia,i...->a...", vs.cf, fB)
    m2 = np.einsum("ia,ib,i...->ab...", vs.cf, vs.cf, fB)
    u = m1 / rho
    eye = np.eye(3).reshape((3, 3) + (1,) * rho.ndim)
    return rho, u, m2 - rho / 3.0 * eye - rho * np.einsum("a...,b...->ab...", u, u)


def _expected_strain(o, geo, face, dn_x):
    """S_ab at the wall nodes of one face (arrays [z, x]) from the closed forms."""
    nz = geo["nz"]
    x = np.arange(NX, dtype=np.float64)[None, :]
    z = np.arange(nz, dtype=np.float64)[:, None]
    s = 1.0 if face == "ymin" else -1.0             # inward direction along y
    S = np.zeros((3, 3, nz, NX))
    # d_y u_x = s * (wall-normal derivative along the inward normal)
    dyux = s * dn_x * np.ones((nz, NX))
    dxuy = geo["e"] * np.cos(geo["kx"] * x) * math.sin(geo["kx"]) * np.ones((nz, NX))
    dzux = geo["g"] * np.cos(geo["kz"] * z) * math.sin(geo["kz"]) * np.ones((nz, NX))
    S[0, 1] = S[1, 0] = 0.5 * (dyux + dxuy)
    S[0, 2] = S[2, 0] = 0.5 * dzux
    return S


def _fd_inward(geo, face):
    """Eq. 28 on the quadratic profile, along the inward normal (exact)."""
    b, c = geo["b"], geo["c"]
    if face == "ymin":
        return b                                     # d/dj at j = 0
    return -(b + 2.0 * c * (NY - 1))                 # -d/dj at j = NY - 1


@pytest.mark.parametrize("beta", [0.0, 0.28, 1.0])
@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_hrfd_rebuilt_moments_match_closed_form(beta, lattice):
    o, f, geo = _setup("wall_hrfd", beta, lattice)
    nt_new = o.nt.copy()
    out = o.hrfd(f.copy(), nt_new)
    vs = o.vs
    d_w = 0.5
    ut = _u_tau(o, geo["U_F"], 1.0 + d_w)
    ypB = ut * d_w / o.nu
    uB = ut * W.u_plus_sa(ypB)
    ana = ut * ut / o.nu * W.dudy_plus_sa(ypB)          # Eq. 15 in lattice units
    nut_B = geo["nt0"] * sa.fv1(geo["nt0"] / o.nu)
    tau = 0.5 + 3.0 * (o.nu + nut_B)
    for face, row in (("ymin", 0), ("ymax", NY - 1)):
        fB = out[:, :, row, :]
        rho, u, neq = _neq_second_moment(vs, fB)
        assert np.allclose(rho, geo["rho_B"], rtol=1e-14)            # Eq. 23
        assert np.allclose(u[0], uB, rtol=1e-12)                     # u_B along t = x
        assert np.abs(u[1]).max() < 1e-16 and np.abs(u[2]).max() < 1e-16
        assert np.allclose(o.utau[face], ut, rtol=1e-12)
        dn = beta * ana + (1.0 - beta) * _fd_inward(geo, face)       # Eq. 27
        S = _expected_strain(o, geo, face, dn)
        if lattice == "D2Q9":
            S[0, 2] = S[2, 0] = 0.0
            S[2, 2] = 0.0
            ref = -2.0 * geo["rho_B"] * tau / 3.0 * S
            ref = ref[:2, :2]
            neq = neq[:2, :2]
        else:
            ref = -2.0 * geo["rho_B"] * tau / 3.0 * S
        # rounding of the O(1/3) second moments is ~1e-16 absolute
        scale = np.abs(ref).max()
        err = np.abs(neq - ref).max()
        assert err <= 1e-12 * scale + 1e-15, (face, err, scale)
        # Dirichlet nu_tilde_B = nu kappa y_B+ (Section 2.2)
        assert np.allclose(nt_new[:, row, :], o.nu * W.KAPPA * ypB, rtol=1e-13)


def test_hrfd_blend_is_linear_in_beta():
    """S_xy is affine in beta with the two ends the analytic (Eq. 15) and the
    finite-difference (Eq. 28) derivatives: S(0.28) = 0.72 S(0) + 0.28 S(1)."""
    vals = {}
    for beta in (0.0, 0.28, 1.0):
        o, f, geo = _setup("wall_hrfd", beta)
        out = o.hrfd(f.copy(), o.nt.copy())
        _, _, neq = _neq_second_moment(o.vs, out[:, :, 0, :])
        vals[beta] = neq[0, 1]
    assert np.allclose(vals[0.28], 0.72 * vals[0.0] + 0.28 * vals[1.0], rtol=1e-12, atol=0)
    # the two ends differ, so the blend is not degenerate on this state
    assert np.abs(vals[1.0] - vals[0.0]).min() > 1e-3 * np.abs(vals[0.0]).max()


def test_cai_degrigny_is_beta_one_with_eq29():
    """Eq. 30: the Cai-Degrigny wall is the beta = 1 wall with the derivative of
    Eq. 29 (the oracle's, pinned by the ratio of Fig. 5) in place of Eq. 15.  As
    Delta+ -> 0 the one-sided difference of Eq. 29 tends to the analytic slope:
    its relative error falls by at least 2^3 per halving of Delta+ (third-order
    difference; near the wall, where u+ ~ y+, the leading term is smaller still)."""
    rel = []
    for U_F in (3.75e-3, 9.375e-4, 2.34375e-4):    # Delta+ ~ 0.5, 0.25, 0.125
        vals = {}
        for scheme in ("wall_cai_degrigny", "wall_hrfd"):
            o, f, geo = _setup(scheme, 1.0, "D2Q9", U_F=U_F, nt0=1e-9)
            o.nu = 1e-2
            out = o.hrfd(f.copy(), o.nt.copy())
            _, _, neq = _neq_second_moment(o.vs, out[:, :, 0, :])
            vals[scheme] = (neq[0, 1], o.utau["ymin"][0, 0])
        (cai, ut), (hr, _) = vals["wall_cai_degrigny"], vals["wall_hrfd"]
        tau = 0.5 + 3.0 * o.nu          # nu_t(1e-9) is negligible: f_v1 ~ chi^3
        x = np.arange(NX, dtype=np.float64)
        e = geo["e"] * np.cos(geo["kx"] * x) * math.sin(geo["kx"])
        # strip the tangential part: what remains is d_y u_x at B
        dcai = 2.0 * cai / (-2.0 * geo["rho_B"] * tau / 3.0) - e
        dhr = 2.0 * hr / (-2.0 * geo["rho_B"] * tau / 3.0) - e
        assert np.allclose(dcai, o.cai_degrigny_derivative(ut), rtol=1e-9)
        assert np.allclose(dhr, ut * ut / o.nu * W.dudy_plus_sa(ut * 0.5 / o.nu), rtol=1e-9)
        rel.append(abs(dcai[0, 0] / dhr[0, 0] - 1.0))
    assert rel[0] > rel[1] * 8 and rel[1] > rel[2] * 8, rel
    assert rel[-1] < 1e-5


def test_hrfd_uses_previous_step_velocity_in_eq28():
    """Eq. 28 differences the previous iteration's velocity field (Section 3.1),
    not the post-stream moments: changing the post-stream populations at F and FF
    (with the same tangential speed at F) leaves the finite-difference part
    unchanged, while changing the stored velocity at FF changes it by exactly
    -(1 - beta)/2 times the change along the inward normal."""
    o, f, geo = _setup("wall_hrfd", 0.0)
    base = o.hrfd(f.copy(), o.nt.copy())
    _, _, n0 = _neq_second_moment(o.vs, base[:, :, 0, :])
    f2 = f.copy()
    f2[:, :, 2, :] = L.equilibrium(o.vs, np.full((geo["nz"], NX), 0.97),
                                   np.stack([np.full((geo["nz"], NX), 0.011),
                                             np.zeros((geo["nz"], NX)),
                                             np.zeros((geo["nz"], NX))]))
    out2 = o.hrfd(f2, o.nt.copy())
    _, _, n2 = _neq_second_moment(o.vs, out2[:, :, 0, :])
    assert np.allclose(n2, n0, rtol=1e-13, atol=0)
    du = 1.0e-3
    o.u[0][:, 2, :] += du
    out3 = o.hrfd(f.copy(), o.nt.copy())
    _, _, n3 = _neq_second_moment(o.vs, out3[:, :, 0, :])
    nut_B = geo["nt0"] * sa.fv1(geo["nt0"] / o.nu)
    tau = 0.5 + 3.0 * (o.nu + nut_B)
    # Eq. 28: -u_FF / 2 per unit change; S_xy = 1/2 d_y u_x
    expect = -2.0 * geo["rho_B"] * tau / 3.0 * 0.5 * (-0.5 * du)
    assert np.allclose(n3[0, 1] - n0[0, 1], expect, rtol=1e-9)
