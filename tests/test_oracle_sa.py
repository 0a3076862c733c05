"""Pins of the oracle's Spalart-Allmaras model (Eqs. 10-14) and stencil.

* closed forms of f_w (Eq. 14) at r = 1 and r -> r_lim;
* c_w1 = c_b1/kappa^2 + (1 + c_b2)/sigma makes the model's right-hand side
  vanish in the log layer (u = u_tau/kappa ln y, nu_tilde = kappa u_tau y,
  d = y): production, destruction and diffusion balance exactly as chi -> oo;
* on linear fields the discrete diffusion and upwind convection are exact.
"""
import numpy as np
import pytest

from oracle import sa


def _pad_linear(a):
    """One ghost layer on every side by linear extrapolation (exact for linear data)."""
    out = np.pad(a, [(0, 0)] * (a.ndim - 3) + [(1, 1)] * 3, mode="edge")
    for ax in range(a.ndim - 3, a.ndim):
        sl_g0 = [slice(None)] * a.ndim
        sl_1 = [slice(None)] * a.ndim
        sl_2 = [slice(None)] * a.ndim
        sl_g0[ax], sl_1[ax], sl_2[ax] = 0, 1, 2
        out[tuple(sl_g0)] = 2 * out[tuple(sl_1)] - out[tuple(sl_2)]
        sl_g1 = [slice(None)] * a.ndim
        sl_m1 = [slice(None)] * a.ndim
        sl_m2 = [slice(None)] * a.ndim
        sl_g1[ax], sl_m1[ax], sl_m2[ax] = -1, -2, -3
        out[tuple(sl_g1)] = 2 * out[tuple(sl_m1)] - out[tuple(sl_m2)]
    return out


def test_fw_closed_forms():
    assert sa.fw(np.array(1.0)) == pytest.approx(1.0, rel=1e-15)
    big = sa.fw(np.array(sa.RLIM))
    assert big == pytest.approx((1 + sa.CW3 ** 6) ** (1 / 6), rel=1e-6)
    assert sa.CW1 == pytest.approx(3.2390678, rel=1e-6)


def test_fv_functions():
    assert sa.fv1(np.array(sa.CV1)) == pytest.approx(0.5)
    assert sa.fv2(np.array(0.0)) == 1.0


def test_log_layer_balance():
    nu = 1e-12                                    # chi -> infinity
    u_tau = 0.05
    ny = 400
    y = np.arange(ny) + 0.5 + 200.0
    shape = (1, ny, 1)
    nt = (sa.KAPPA * u_tau * y).reshape(shape)
    u = np.zeros((3,) + shape)
    u[0] = (u_tau / sa.KAPPA * np.log(y)).reshape(shape)
    inv_d2 = (1.0 / y ** 2).reshape(shape)
    # periodic x and z (size 1), linear ghosts in y for nu_tilde; log ghosts for u
    ntp = np.pad(nt, 1, mode="wrap")
    ntp[:, 0, :] = 2 * ntp[:, 1, :] - ntp[:, 2, :]
    ntp[:, -1, :] = 2 * ntp[:, -2, :] - ntp[:, -3, :]
    up = np.pad(u, ((0, 0), (1, 1), (1, 1), (1, 1)), mode="wrap")
    yg = np.concatenate([[y[0] - 1], y, [y[-1] + 1]])
    up[0, :, :, :] = (u_tau / sa.KAPPA * np.log(yg))[None, :, None]
    r = sa.rhs(ntp, up, nu, inv_d2).ravel() / (sa.CB1 * u_tau ** 2)
    # the residual is the O(1/y^2) truncation of the central vorticity stencil
    # (|S_h - S| / S = 1/(3 y^2)) carried into r and f_w: small and decaying as 1/y^2
    assert np.abs(r).max() < 2e-4
    ratio = (r[0] * y[0] ** 2) / (r[-1] * y[-1] ** 2)
    assert ratio == pytest.approx(1.0, rel=0.02)
    # a dropped term would leave an O(1) imbalance
    assert abs(sa.CB1 * u_tau ** 2 - sa.CW1 * sa.KAPPA ** 2 * u_tau ** 2
               + (1 + sa.CB2) * sa.KAPPA ** 2 * u_tau ** 2 / sa.SIGMA) < 1e-16


def test_linear_fields_exact():
    rng = np.random.default_rng(5)
    shape = (4, 5, 6)
    z, y, x = np.meshgrid(np.arange(4), np.arange(5), np.arange(6), indexing="ij")
    g = np.array([2e-4, -3e-4, 1e-4])                   # d nt / d(x, y, z)
    nt = 0.05 + g[0] * x + g[1] * y + g[2] * z
    U = np.array([0.03, -0.02, 0.01])
    u = np.broadcast_to(U[:, None, None, None], (3,) + shape).copy()
    nu = 1e-3
    r = sa.rhs(_pad_linear(nt), _pad_linear(u), nu, np.zeros(shape))
    # S = 0 (uniform u) and 1/d^2 = 0: no production or destruction
    conv = (U * g).sum()
    ref = -conv + (1.0 + sa.CB2) * (g * g).sum() / sa.SIGMA
    assert np.allclose(r, ref, rtol=1e-12, atol=1e-18)
    del rng


def test_vorticity_of_rigid_rotation():
    # u = Omega x r about z: |curl u| = 2 Omega exactly with central differences
    shape = (3, 6, 7)
    z, y, x = np.meshgrid(np.arange(3), np.arange(6), np.arange(7), indexing="ij")
    Om = 1e-3
    u = np.stack([-Om * y, Om * x, 0.0 * x]).astype(np.float64)
    nt = np.full(shape, 1e-3)
    nu = 1.0
    # with nu huge, chi is tiny: f_v1 ~ 0, f_v2 ~ 1, Sbar ~ nt / (kappa^2 d^2)
    inv_d2 = np.zeros(shape)
    r = sa.rhs(_pad_linear(nt), _pad_linear(u), nu, inv_d2)
    # P = c_b1 * S~ * nt with S~ = S = 2 Omega; D = 0; no diffusion; convection 0
    assert np.allclose(r, sa.CB1 * 2 * Om * 1e-3, rtol=1e-12)


def _sbar_state(sbar_over_S, S=2e-3, nu=1e-4):
    """(nt, S, nu, inv_d2) with Sbar = nt f_v2 / (kappa d)^2 equal to sbar_over_S * S:
    chi = 10 makes f_v2 negative, and 1/d^2 is solved for."""
    nt = 10.0 * nu
    fv2 = sa.fv2(np.array(10.0))
    assert fv2 < 0
    inv_d2 = sbar_over_S * S * sa.KAPPA ** 2 / (nt * fv2)
    return nt, S, nu, inv_d2


def test_s_tilde_limiter_second_branch():
    """Eq. 13 with the ICCFD7 limiter (c_v2 = 0.7, c_v3 = 0.9) where Sbar < -c_v2 S:
    the branch meets S + Sbar = (1 - c_v2) S = 0.3 S at the switch, equals
    S (1 + (c_v2^2 - c_v3) / (c_v3 - 2 c_v2 + 1)) = 0.18 S at Sbar = -S, tends to
    (1 - c_v3) S = 0.1 S as Sbar -> -inf and stays positive and increasing."""
    S = 2e-3
    st = lambda k: float(sa.s_tilde(*_sbar_state(k, S)))  # noqa: E731
    assert st(-0.7) == pytest.approx(0.3 * S, rel=1e-12)
    assert st(-0.7 - 1e-9) == pytest.approx(0.3 * S, rel=1e-7)
    assert st(-0.7 + 1e-9) == pytest.approx(0.3 * S, rel=1e-7)
    assert st(-1.0) == pytest.approx(0.18 * S, rel=1e-12)
    assert st(-1e8) == pytest.approx(0.1 * S, rel=1e-6)
    ks = -np.logspace(np.log10(0.7), 6, 200)
    vals = np.array([st(k) for k in ks])
    assert np.all(vals > 0.1 * S) and np.all(np.diff(vals) < 0)
    # the first branch, S + Sbar, is untouched above the switch
    assert st(-0.5) == pytest.approx(0.5 * S, rel=1e-12)
    assert st(2.0) == pytest.approx(3.0 * S, rel=1e-12)


def test_source_uses_the_limited_s_tilde():
    """P of Eq. 12 is c_b1 S~ nu_tilde on the limited branch, and r of Eq. 14 is
    taken with the limited S~: at Sbar = -S (S~ = 0.18 S) the source equals
    c_b1 0.18 S nt - c_w1 f_w(r) nt^2 / d^2 with r = min(nt / (0.18 S kappa^2 d^2), 10)."""
    S = 2e-3
    nt, S, nu, inv_d2 = _sbar_state(-1.0, S)
    r = min(nt * inv_d2 / (sa.KAPPA ** 2 * 0.18 * S), sa.RLIM)
    ref = sa.CB1 * 0.18 * S * nt - sa.CW1 * float(sa.fw(np.array(r))) * nt * nt * inv_d2
    assert float(sa.source(np.array(nt), np.array(S), nu, np.array(inv_d2))) == \
        pytest.approx(ref, rel=1e-12)
