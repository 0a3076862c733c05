"""Wall functions and the friction-velocity inversion (oracle, FP64).

Test infrastructure only (see the package docstring).

* Eq. 15: the SA-consistent law-of-the-wall slope
      du+/dy+ = (c_v1^3 + (kappa y+)^3) / (c_v1^3 + (1 + kappa y+) (kappa y+)^3).
* Eq. 16: its analytic integral with u+(0) = 0, constants printed in Section 2.2.
  The printed arctan(b/(y+ + a)) jumps by pi at y+ = -a_2 = 6.93 (a_2 < 0); the
  continuous branch atan2(b, y+ + a) is used, which equals the printed form for
  y+ > 6.93 and makes d(Eq. 16)/dy+ equal Eq. 15 everywhere.
* Log law u+ = ln(y+) / kappa + B (the law the first-node tests enforce).
* Newton-Raphson for u_tau from U = u_tau u+(u_tau y / nu) (Section 3.1), with a
  bisection safeguard so every iterate stays inside a sign-change bracket.
"""
from __future__ import annotations

import numpy as np

KAPPA = 0.41
CV1 = 7.1

# Eq. 16 constants (Section 2.2)
B_BAR = 5.033908790505579
A1 = 8.148221580024245
A2 = -6.9287093849022945
B1 = 7.4600876082527945
B2 = 7.468145790401841
C1 = 2.5496773539754747
C2 = 1.3301651588535228
C3 = 3.599459109332379
C4 = 3.639753186868684494


def dudy_plus_sa(yp):
    """Eq. 15: du+/dy+ of the SA-consistent wall function."""
    ky = KAPPA * np.asarray(yp, dtype=np.float64)
    return (CV1 ** 3 + ky ** 3) / (CV1 ** 3 + (1.0 + ky) * ky ** 3)


def u_plus_sa(yp):
    """Eq. 16 (continuous atan2 branch)."""
    y = np.asarray(yp, dtype=np.float64)
    return (B_BAR + C1 * np.log((y + A1) ** 2 + B1 ** 2)
            - C2 * np.log((y + A2) ** 2 + B2 ** 2)
            - C3 * np.arctan2(B1, y + A1) - C4 * np.arctan2(B2, y + A2))


def u_plus_log(yp, kappa=KAPPA, B=5.2):
    """Log law u+ = ln(y+)/kappa + B."""
    return np.log(np.asarray(yp, dtype=np.float64)) / kappa + B


def dudy_plus_log(yp, kappa=KAPPA):
    return 1.0 / (kappa * np.asarray(yp, dtype=np.float64))


class WallLaw:
    """Selects Eq. 16 ("sa_analytic") or the log law ("log")."""

    def __init__(self, kind="sa_analytic", kappa=KAPPA, B=5.2):
        self.kind, self.kappa, self.B = kind, kappa, B

    def u_plus(self, yp):
        if self.kind == "sa_analytic":
            return u_plus_sa(yp)
        return u_plus_log(yp, self.kappa, self.B)

    def dudy_plus(self, yp):
        if self.kind == "sa_analytic":
            return dudy_plus_sa(yp)
        return dudy_plus_log(yp, self.kappa)


def solve_u_tau(law: WallLaw, U, y, nu, max_iter=200):
    """Solve U = u_tau * u+(u_tau y / nu) for u_tau >= 0, elementwise.

    U >= 0 (tangential speed at the reference node), y > 0 its wall distance.
    U == 0 gives u_tau = 0.  G(u) = u u+(u y/nu) - U is increasing (Eq. 16) or
    convex with G(0+) = -U (log law), so the positive root is unique; the
    iteration keeps a bracket [lo, hi] with G(lo) < 0 < G(hi) and takes the Newton
    step when it stays inside, else bisects, until the step is below 1e-15 u_tau.
    Parity pinned by the round trip U -> u_tau -> U.
    """
    U = np.atleast_1d(np.asarray(U, dtype=np.float64)).copy()
    out = np.zeros_like(U)
    act = U > 0.0
    if not act.any():
        return out
    Ua = U[act]

    def G(u):
        yp = u * y / nu
        return u * law.u_plus(yp) - Ua, law.u_plus(yp) + yp * law.dudy_plus(yp)

    lo = np.zeros_like(Ua)
    hi = np.maximum(Ua, np.sqrt(Ua * nu / y))
    for _ in range(400):
        g, _ = G(hi)
        grow = g <= 0.0
        if not grow.any():
            break
        hi = np.where(grow, 2.0 * hi, hi)
    x = 0.5 * (lo + hi)
    done = np.zeros(Ua.shape, dtype=bool)
    for _ in range(max_iter):
        g, dg = G(x)
        lo = np.where(g < 0.0, x, lo)
        hi = np.where(g > 0.0, x, hi)
        with np.errstate(divide="ignore", invalid="ignore"):
            xn = x - g / dg
        bad = ~((xn > lo) & (xn < hi)) | ~np.isfinite(xn)
        xn = np.where(bad, 0.5 * (lo + hi), xn)
        step = np.abs(xn - x)
        done_now = (step <= 1e-15 * np.abs(xn)) | (g == 0.0)
        x = np.where(done, x, xn)
        done |= done_now
        if done.all():
            break
    out[act] = x
    return out
