"""Pins of the oracle's lattice tables and local collision operators.

Each check follows from the lattice's isotropy or from moment identities that
hold exactly for the operators of Section 2.1 (Eqs. 2-6, 8), not from the
oracle's own formulas.
"""
import itertools

import numpy as np
import pytest

from oracle import lattice as L

SETS = ["D2Q9", "D3Q19"]


def _delta(a, b):
    return 1.0 if a == b else 0.0


@pytest.mark.parametrize("name", SETS)
def test_isotropy(name):
    vs = L.VelocitySet(name)
    dim = 2 if name == "D2Q9" else 3
    assert vs.q == (9 if name == "D2Q9" else 19)
    assert abs(vs.w.sum() - 1.0) < 1e-15
    c = vs.cf[:, :dim]
    assert np.abs(vs.w @ c).max() < 1e-15
    second = np.einsum("i,ia,ib->ab", vs.w, c, c)
    assert np.allclose(second, np.eye(dim) / 3.0, atol=1e-15)
    third = np.einsum("i,ia,ib,ic->abc", vs.w, c, c, c)
    assert np.abs(third).max() < 1e-15
    fourth = np.einsum("i,ia,ib,ic,id->abcd", vs.w, c, c, c, c)
    for a, b, cc, d in itertools.product(range(dim), repeat=4):
        ref = (_delta(a, b) * _delta(cc, d) + _delta(a, cc) * _delta(b, d)
               + _delta(a, d) * _delta(b, cc)) / 9.0
        assert abs(fourth[a, b, cc, d] - ref) < 1e-15


@pytest.mark.parametrize("name", SETS)
def test_opposite_and_mirror(name):
    vs = L.VelocitySet(name)
    assert (vs.c[vs.opp] == -vs.c).all()
    for ax in range(3):
        m = vs.mirror(ax)
        ref = vs.c.copy()
        ref[:, ax] *= -1
        assert (vs.c[m] == ref).all()


def _random_state(vs, rng, shape=(2, 3, 4)):
    rho = 1.0 + 0.05 * rng.standard_normal(shape)
    u = 0.05 * rng.standard_normal((3,) + shape)
    if vs.name == "D2Q9":
        u[2] = 0.0
    return rho, u


@pytest.mark.parametrize("name", SETS)
def test_equilibrium_moments(name):
    vs = L.VelocitySet(name)
    rng = np.random.default_rng(1)
    rho, u = _random_state(vs, rng)
    feq = L.equilibrium(vs, rho, u)
    assert np.allclose(feq.sum(0), rho, rtol=1e-14)
    mom = np.einsum("ia,i...->a...", vs.cf, feq)
    assert np.allclose(mom, rho * u, atol=1e-15)
    pi = np.einsum("ia,ib,i...->ab...", vs.cf, vs.cf, feq)
    ref = rho * (np.eye(3)[:, :, None, None, None] / 3.0) + rho * np.einsum("a...,b...->ab...", u, u)
    dim = 2 if name == "D2Q9" else 3
    assert np.allclose(pi[:dim, :dim], ref[:dim, :dim], atol=1e-15)


@pytest.mark.parametrize("name", SETS)
def test_guo_force_moments(name):
    vs = L.VelocitySet(name)
    rng = np.random.default_rng(2)
    rho, u = _random_state(vs, rng)
    F = np.array([1e-3, -2e-3, 0.0 if name == "D2Q9" else 5e-4])
    Fi = L.guo_force(vs, u, F)
    assert np.abs(Fi.sum(0)).max() < 1e-17
    m1 = np.einsum("ia,i...->a...", vs.cf, Fi)
    assert np.allclose(m1, F[:, None, None, None], atol=1e-17)
    m2 = np.einsum("ia,ib,i...->ab...", vs.cf, vs.cf, Fi)
    ref = np.einsum("a...,b->ab...", u, F) + np.einsum("a,b...->ab...", F, u)
    dim = 2 if name == "D2Q9" else 3
    assert np.allclose(m2[:dim, :dim], ref[:dim, :dim], atol=1e-17)


@pytest.mark.parametrize("name", SETS)
@pytest.mark.parametrize("op", ["bgk", "regularized"])
def test_collision_conservation_and_relaxation(name, op):
    """Mass conserved, momentum raised by F, and the non-equilibrium second
    moment relaxed by (1 - omega) (the Chapman-Enskog content of Eq. 8)."""
    vs = L.VelocitySet(name)
    rng = np.random.default_rng(3)
    rho, u = _random_state(vs, rng)
    f = L.equilibrium(vs, rho, u) * (1.0 + 0.02 * rng.standard_normal((vs.q,) + rho.shape))
    F = np.array([1e-4, 2e-4, 0.0])
    rho_m, u_m = L.moments(vs, f, F)
    omega = 1.0 / (0.5 + 3.0 * (0.01 + 0.05 * rng.random(rho.shape)))
    coll = L.collide_bgk if op == "bgk" else L.collide_regularized
    fs = coll(vs, f, rho_m, u_m, omega, F)
    assert np.allclose(fs.sum(0), f.sum(0), rtol=1e-14)
    mom_in = np.einsum("ia,i...->a...", vs.cf, f)
    mom_out = np.einsum("ia,i...->a...", vs.cf, fs)
    assert np.allclose(mom_out - mom_in, F[:, None, None, None], atol=1e-15)
    feq = L.equilibrium(vs, rho_m, u_m)
    pin = np.einsum("ia,ib,i...->ab...", vs.cf, vs.cf, f - feq)
    pout = np.einsum("ia,ib,i...->ab...", vs.cf, vs.cf, fs - feq)
    Fi = L.guo_force(vs, u_m, F)
    pf = np.einsum("ia,ib,i...->ab...", vs.cf, vs.cf, Fi) * (1.0 - 0.5 * omega)
    dim = 2 if name == "D2Q9" else 3
    assert np.allclose(pout[:dim, :dim], ((1.0 - omega) * pin + pf)[:dim, :dim], atol=1e-14)


def test_omega_eq8():
    # Eq. 8 with c_s^2 = 1/3: omega = 1 at nu = 1/6, omega -> 2 as nu -> 0
    assert L.omega_from_viscosity(1.0 / 6.0) == pytest.approx(1.0, abs=1e-15)
    assert L.omega_from_viscosity(0.0) == pytest.approx(2.0)
