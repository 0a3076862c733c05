"""Lattice velocity sets and local collision operators (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 2.1: populations f_i stream along discrete velocities c_i (Eq. 3) and
relax locally (Eq. 2); density and velocity are the zeroth and first moments
with the half-force shift of Eq. 5; the relaxation frequency follows from the
effective viscosity through Eq. 8, omega = 1 / (1/2 + nu_eff / c_s^2), c_s^2 = 1/3.

The paper's collision is de Rosis' central-moment operator (Eq. 7), whose
transform matrix and fourth-order equilibrium are not printed in the paper.  As
its substitutes this oracle implements the two operators the method is run
with here: BGK with the second-order Hermite equilibrium and Guo forcing, and
the regularized BGK that projects the non-equilibrium part onto its
second-order Hermite moment.
"""
from __future__ import annotations

import itertools

import numpy as np

CS2 = 1.0 / 3.0


class VelocitySet:
    """D2Q9 or D3Q19: every c in {-1,0,1}^D with |c|^2 <= 2 (2-D sets carry c_z = 0).

    Weights by |c|^2: D2Q9 (4/9, 1/9, 1/36), D3Q19 (1/3, 1/18, 1/36).
    Pinned by the lattice isotropy conditions up to fourth order.
    """

    def __init__(self, name: str):
        self.name = name
        if name == "D2Q9":
            vecs = [(a, b, 0) for a, b in itertools.product((-1, 0, 1), repeat=2)]
            wmap = {0: 4.0 / 9.0, 1: 1.0 / 9.0, 2: 1.0 / 36.0}
        elif name == "D3Q19":
            vecs = [v for v in itertools.product((-1, 0, 1), repeat=3)
                    if sum(x * x for x in v) <= 2]
            wmap = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}
        else:
            raise ValueError(name)
        vecs.sort(key=lambda v: (sum(x * x for x in v), v))
        self.c = np.array(vecs, dtype=np.int64)            # (Q, 3)
        self.q = len(vecs)
        self.w = np.array([wmap[int((v * v).sum())] for v in self.c])
        self.cf = self.c.astype(np.float64)
        index = {tuple(v): i for i, v in enumerate(vecs)}
        self.opp = np.array([index[tuple(-v)] for v in self.c])

    def mirror(self, axis: int) -> np.ndarray:
        """Index of the velocity with component ``axis`` negated (specular reflection)."""
        index = {tuple(v): i for i, v in enumerate(self.c.tolist())}
        out = []
        for v in self.c.tolist():
            m = list(v)
            m[axis] = -m[axis]
            out.append(index[tuple(m)])
        return np.array(out)


def _bcast(v, ndim):
    return v.reshape(v.shape + (1,) * ndim)


def equilibrium(vs: VelocitySet, rho, u):
    """Second-order Hermite equilibrium f_i^eq = w_i rho (1 + c.u/cs^2 + (c.u)^2/(2 cs^4) - u.u/(2 cs^2)).

    ``rho`` has shape S, ``u`` (3,)+S; returns (Q,)+S.
    """
    cu = np.tensordot(vs.cf, u, axes=(1, 0))               # (Q,)+S
    uu = (u * u).sum(axis=0)
    w = _bcast(vs.w, rho.ndim)
    return w * rho * (1.0 + cu / CS2 + 0.5 * cu * cu / (CS2 * CS2) - 0.5 * uu / CS2)


def guo_force(vs: VelocitySet, u, F):
    """Guo et al. forcing term F_i = w_i [(c_i - u)/cs^2 + (c_i.u) c_i / cs^4] . F.

    ``F`` is a 3-vector (constant force density); returns (Q,)+S.  Its zeroth
    moment is 0 and its first moment is F, consistent with the half-force
    velocity of Eq. 5.
    """
    F = np.asarray(F, dtype=np.float64)
    S = u.shape[1:]
    cF = vs.cf @ F                                          # (Q,)
    uF = np.tensordot(F, u, axes=(0, 0))                    # S
    cu = np.tensordot(vs.cf, u, axes=(1, 0))                # (Q,)+S
    w = _bcast(vs.w, len(S))
    return w * ((_bcast(cF, len(S)) - uF[None]) / CS2 + cu * _bcast(cF, len(S)) / (CS2 * CS2))


def moments(vs: VelocitySet, f, F):
    """rho = sum_i f_i (Eq. 4); rho u = sum_i f_i c_i + F/2 (Eq. 5)."""
    rho = f.sum(axis=0)
    mom = np.tensordot(vs.cf.T, f, axes=(1, 0))             # (3,)+S
    F = np.asarray(F, dtype=np.float64)
    u = (mom + _bcast(F, rho.ndim) * 0.5) / rho[None]
    return rho, u


def omega_from_viscosity(nu_eff):
    """Eq. 8 with nu replaced by nu_eff = nu + nu_t: omega = (1/2 + nu_eff / cs^2)^-1."""
    return 1.0 / (0.5 + nu_eff / CS2)


def second_order_Q(vs: VelocitySet):
    """Q_i,ab = c_ia c_ib - cs^2 delta_ab, shape (Q, 3, 3) (defined under Eq. 18)."""
    return np.einsum("ia,ib->iab", vs.cf, vs.cf) - CS2 * np.eye(3)[None]


def collide_bgk(vs: VelocitySet, f, rho, u, omega, F):
    """BGK with Guo forcing: f* = f - omega (f - f^eq) + (1 - omega/2) F_i."""
    feq = equilibrium(vs, rho, u)
    return f - omega[None] * (f - feq) + (1.0 - 0.5 * omega[None]) * guo_force(vs, u, F)


def collide_regularized(vs: VelocitySet, f, rho, u, omega, F):
    """Regularized BGK: f* = f^eq + (1 - omega) P(f - f^eq) + (1 - omega/2) F_i.

    P is the Hermite projection of the non-equilibrium part up to second order,
    P(g)_i = w_i [c_i . a1 / cs^2 + Q_i : Pi / (2 cs^4)] with a1 = sum_i g_i c_i and
    Pi = sum_i g_i c_i c_i (its zeroth moment vanishes).  Under Guo forcing
    a1 = -F/2, so keeping it makes the moments up to second order those of BGK.
    """
    feq = equilibrium(vs, rho, u)
    neq = f - feq
    a1 = np.tensordot(vs.cf.T, neq, axes=(1, 0))            # (3,)+S
    pi = np.einsum("ia,ib,i...->ab...", vs.cf, vs.cf, neq)  # (3,3)+S
    Q = second_order_Q(vs)
    w = _bcast(vs.w, rho.ndim)
    f1 = w * (np.tensordot(vs.cf, a1, axes=(1, 0)) / CS2
              + np.einsum("iab,ab...->i...", Q, pi) / (2.0 * CS2 * CS2))
    return feq + (1.0 - omega[None]) * f1 + (1.0 - 0.5 * omega[None]) * guo_force(vs, u, F)
