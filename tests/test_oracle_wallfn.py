"""Pins of the wall functions, the u_tau inversion and the SA wall identity.

* Eq. 16 is checked against a quadrature of Eq. 15 (scipy), which is what the
  paper says it is: the analytic integral of Eq. 15 with u+(0) = 0.
* Its logarithmic asymptote ln(y+)/kappa + B_bar follows from the constants.
* Eq. 15 combined with Eq. 10 gives the exact identity
  (1 + nu_t/nu) du+/dy+ = 1 when nu_tilde = nu kappa y+ (the Dirichlet value of
  Section 2.2): the wall function carries a constant total shear stress (Eq. 33).
"""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import sa, wallfn as W


def test_eq16_is_integral_of_eq15():
    u0 = W.u_plus_sa(0.0)
    assert abs(u0) < 1e-3                     # u_WF(0) = 0 up to the printed constants
    for y in [0.5, 3.0, 6.9, 7.0, 11.0, 30.0, 100.0, 1000.0, 2e4]:
        val, _ = quad(lambda t: float(W.dudy_plus_sa(t)), 0.0, y, limit=400,
                      epsabs=1e-13, epsrel=1e-13)
        assert W.u_plus_sa(y) - u0 == pytest.approx(val, rel=1e-10, abs=1e-10)


def test_eq16_continuous_across_minus_a2():
    y = -W.A2
    assert abs(W.u_plus_sa(y + 1e-9) - W.u_plus_sa(y - 1e-9)) < 1e-8


def test_eq16_asymptote():
    assert 2.0 * (W.C1 - W.C2) == pytest.approx(1.0 / W.KAPPA, rel=1e-14)
    y = 1e9
    assert W.u_plus_sa(y) - np.log(y) / W.KAPPA == pytest.approx(W.B_BAR, abs=1e-7)


def test_sa_wall_identity():
    yp = np.logspace(-2, 5, 200)
    nu = 1.0
    nut = sa.nu_t(nu * W.KAPPA * yp, nu)
    assert np.allclose((1.0 + nut / nu) * W.dudy_plus_sa(yp), 1.0, rtol=1e-13)


@pytest.mark.parametrize("kind", ["sa_analytic", "log"])
def test_newton_round_trip(kind):
    law = W.WallLaw(kind, 0.41, 5.2)
    nu = 1.5e-5
    for y in [0.0125, 0.075, 0.3]:
        ut = np.array([0.0, 1e-4, 0.01, 0.063, 0.3, 2.0])
        U = ut * law.u_plus(ut * y / nu)
        U[0] = 0.0
        got = W.solve_u_tau(law, U, y, nu)
        ok = U > 0
        assert got[0] == 0.0
        assert np.allclose(got[ok], ut[ok], rtol=1e-14)


def test_newton_example_channel():
    # Re_tau = 4200 channel: u_tau = 0.063, reference node at y_F = 0.075
    law = W.WallLaw("sa_analytic")
    U = 0.063 * W.u_plus_sa(0.063 * 0.075 / 1.5e-5)
    assert W.solve_u_tau(law, np.array([U]), 0.075, 1.5e-5)[0] == pytest.approx(0.063, rel=1e-15)


def test_log_law_values():
    # u+ = ln(y+)/kappa + B: at y+ = e^(-kappa B) the law crosses zero
    law = W.WallLaw("log", 0.41, 5.2)
    assert law.u_plus(np.exp(-0.41 * 5.2)) == pytest.approx(0.0, abs=1e-14)
    assert law.u_plus(np.e) == pytest.approx(1.0 / 0.41 + 5.2, rel=1e-15)
