"""Spalart-Allmaras one-equation model (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 2.2, Eqs. 10-14, baseline SA with the constants printed there.  The
paper fixes the discretisation only in words: vorticity by second-order central
differences of the LBM velocity, convection first-order upwind, diffusion with
standard second-order differences.  Readings taken where it is silent:

* explicit Euler in time with the lattice step (dt = 1, dx = 1);
* diffusion written conservatively, d/dx((nu + nt) d nt/dx) with face values of
  nt the arithmetic mean of the two cells; the c_b2 |grad nt|^2 term with central
  differences; upwinding by the sign of the cell's own velocity component;
* the modified vorticity is kept positive with the continuous limiter of
  Allmaras, Johnson & Spalart (ICCFD7, 2012): S~ = S + Sbar if Sbar >= -c_v2 S,
  else S + S (c_v2^2 S + c_v3 Sbar) / ((c_v3 - 2 c_v2) S - Sbar), c_v2 = 0.7,
  c_v3 = 0.9; r = r_lim where S~ <= 0; nt is clipped at 0 after the update.
"""
from __future__ import annotations

import numpy as np

CB1 = 0.1355
CB2 = 0.622
SIGMA = 2.0 / 3.0
KAPPA = 0.41
CW1 = CB1 / KAPPA ** 2 + (1.0 + CB2) / SIGMA
CW2 = 0.3
CW3 = 2.0
CV1 = 7.1
RLIM = 10.0
CV2_LIM = 0.7
CV3_LIM = 0.9


def fv1(chi):
    """Eq. 10: f_v1 = chi^3 / (chi^3 + c_v1^3)."""
    c3 = chi ** 3
    return c3 / (c3 + CV1 ** 3)


def fv2(chi):
    """Eq. 13: f_v2 = 1 - chi / (1 + chi f_v1)."""
    return 1.0 - chi / (1.0 + chi * fv1(chi))


def fw(r):
    """Eq. 14: f_w = g ((1 + c_w3^6) / (g^6 + c_w3^6))^(1/6), g = r + c_w2 (r^6 - r)."""
    g = r + CW2 * (r ** 6 - r)
    return g * ((1.0 + CW3 ** 6) / (g ** 6 + CW3 ** 6)) ** (1.0 / 6.0)


def nu_t(nt, nu):
    """Eq. 10: nu_t = nu_tilde f_v1(nu_tilde / nu)."""
    return nt * fv1(nt / nu)


def s_tilde(nt, S, nu, inv_d2):
    """Modified vorticity of Eq. 13, S~ = S + Sbar with Sbar = nu_tilde f_v2 / (kappa d)^2,
    kept positive by the ICCFD7 limiter: where Sbar < -c_v2 S the value is
    S + S (c_v2^2 S + c_v3 Sbar) / ((c_v3 - 2 c_v2) S - Sbar), which meets S + Sbar at
    Sbar = -c_v2 S and tends to (1 - c_v3) S as Sbar -> -inf."""
    chi = nt / nu
    sbar = nt * fv2(chi) * (inv_d2 / KAPPA ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        lim = S + S * (CV2_LIM ** 2 * S + CV3_LIM * sbar) / ((CV3_LIM - 2.0 * CV2_LIM) * S - sbar)
    return np.where(sbar >= -CV2_LIM * S, S + sbar, lim)


def source(nt, S, nu, inv_d2):
    """P - D of Eq. 12 with S~ of Eq. 13 and r of Eq. 14.

    ``S`` is the vorticity magnitude, ``inv_d2`` = 1 / d^2 (0 with no wall).
    """
    inv_kd2 = inv_d2 / KAPPA ** 2
    st = s_tilde(nt, S, nu, inv_d2)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(st > 0.0, np.minimum(nt * inv_kd2 / st, RLIM), RLIM)
    P = CB1 * st * nt
    D = CW1 * fw(r) * nt * nt * inv_d2
    return P - D


def _nb(a, axis_xyz, s):
    """Neighbour field at offset s (+1/-1) along x/y/z for the interior of a padded
    array indexed [..., z, y, x] with one ghost layer on every side."""
    nd = a.ndim
    sl = [slice(None)] * (nd - 3) + [slice(1, -1)] * 3
    ax = nd - 1 - axis_xyz
    n = a.shape[ax] - 2
    sl[ax] = slice(1 + s, 1 + s + n)
    return a[tuple(sl)]


def rhs(nt_pad, u_pad, nu, inv_d2):
    """Right-hand side of Eq. 11 on the interior cells.

    ``nt_pad`` is nu_tilde with one ghost layer, ``u_pad`` the velocity (3, ...)
    with one ghost layer; lattice units.
    """
    nt = _nb(nt_pad, 0, 0)
    u = _nb(u_pad, 0, 0)
    # vorticity by central differences: d_a u_g = (u_g(+a) - u_g(-a)) / 2
    def d(g, a):
        return 0.5 * (_nb(u_pad[g], a, 1) - _nb(u_pad[g], a, -1))
    wx = d(2, 1) - d(1, 2)
    wy = d(0, 2) - d(2, 0)
    wz = d(1, 0) - d(0, 1)
    S = np.sqrt(wx * wx + wy * wy + wz * wz)
    conv = np.zeros_like(nt)
    diff = np.zeros_like(nt)
    grad2 = np.zeros_like(nt)
    for a in range(3):
        ntp = _nb(nt_pad, a, 1)
        ntm = _nb(nt_pad, a, -1)
        ua = u[a]
        conv += np.where(ua > 0.0, ua * (nt - ntm), ua * (ntp - nt))
        diff += (nu + 0.5 * (nt + ntp)) * (ntp - nt) - (nu + 0.5 * (nt + ntm)) * (nt - ntm)
        grad2 += (0.5 * (ntp - ntm)) ** 2
    return -conv + source(nt, S, nu, inv_d2) + (diff + CB2 * grad2) / SIGMA
