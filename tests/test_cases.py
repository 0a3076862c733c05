"""The seeded workload definitions (lbm_cases): the stated recipes for the
initial fields and the wall rules, checked on small instances."""
import numpy as np

import lbm_cases as C


def test_channel_log_layer_start():
    """3-D channel: nu_tilde = max(3 nu, kappa u_tau d), d the distance to the
    nearer wall with the boundary nodes d_w Delta from it; velocity U_b with the
    seeded +/- 1 % perturbation; Delta = 2h / (ny - 1 + 2 d_w)."""
    for d_w in (0.5, 0.3):
        c = C.channel_3d(re_tau=5200.0, nx=8, ny=16, nz=2, d_w=d_w, interp="yu")
        assert np.isclose(c.dx, 2.0 / (16 - 1 + 2 * d_w))
        rho, u, nt = C.initial_fields(c)
        par = C.channel_parameters(5200.0)
        j = np.arange(16.0)
        d = np.minimum(j + d_w, 15 - j + d_w) * c.dx
        ref = np.maximum(3.0 * c.nu, c.kappa * par["u_tau"] * d)
        assert np.allclose(nt[0, :, 0], ref, rtol=1e-15)
        assert np.all(nt == nt[:, :, :1])                  # uniform along x and z
        assert np.all(np.abs(u[0] / par["u_b"] - 1.0) <= 0.01 + 1e-15)
        assert np.all(u[1] == 0.0) and np.all(rho == c.rho0)
    uni = C.channel_3d(nx=4, ny=8, nz=1, nut_init="uniform").replace(lattice="D2Q9")
    assert np.all(C.initial_fields(uni)[2] == 3.0 * uni.nu)


def test_plate_wall_rule_defaults():
    """The plate's bounce-back wall uses Yu's rule (the paper's choice on the
    plate); regularized walls take no interpolation; half-way stays selectable."""
    assert C.flat_plate_3d(nx=8, ny=8, nz=1).bcs["ymin"].interp == "yu"
    assert C.flat_plate_3d(nx=8, ny=8, nz=1, scheme="wall_hrfd").bcs["ymin"].interp == "none"
    assert C.flat_plate_3d(nx=8, ny=8, nz=1, interp="none").bcs["ymin"].interp == "none"
    # the plate starts uniform: nu_tilde = 3 nu everywhere
    c = C.flat_plate_3d(nx=8, ny=8, nz=1).replace(lattice="D2Q9")
    assert np.all(C.initial_fields(c)[2] == 3.0 * c.nu)


def test_batched_sweep_is_seeded_and_shardable():
    a = C.batched_sweep(96)
    b = C.batched_sweep(96)
    assert [x.name for x in a] == [x.name for x in b]
    assert {x.lattice for x in a} == {"D2Q9", "D3Q19"}
    cells = [x.cells for x in a]
    parts = [C.shard_instances(cells, 3, r) for r in range(3)]
    assert sorted(i for p in parts for i in p) == list(range(96))
