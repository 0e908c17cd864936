"""Per-node virtual wall density (lbm_set_wall_density; the oracle's or_set_wall_density).

Sec. 3 gives every wall psi(rho_s) with one virtual density rho_s (Benzi et al.'s
virtual-density walls).  A field of wall densities sets it node by node, so that different
walls can be wetted by different phases (the annular shear flow of Sec. 3.2 needs gas at the
inner cylinder and liquid at the outer one).

Pins on the oracle: a uniform field equal to rho_s reproduces the scalar walls bit for bit;
the lattice's mirror symmetry maps a channel with wall densities (A below, B above) onto
the one with (B below, A above); and a liquid-like wall raises the density of the gas next
to it above that next to a gas-like wall (the sign of the wetting).  A wall far denser
than the phase against it (rho_s near rho_l against gas) pulls that phase so hard that the
density leaves the range where psi is real: the tests keep rho_s <= 0.3 rho_l against gas.
The GPU parity of the same feature is in test_gpu_wall_density.py."""
import numpy as np

from oracle import oracle as O
from paper_2604_13407_gb300 import inputs as I
from tests.setups import cs_case, cs_params


def channel(nx=8, ny=40):
    """Periodic in x and y, solid rows at y = 0 and y = ny - 1, a liquid slab between gas
    layers at the walls."""
    T, rg, rl = cs_case()
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[-1, :] = 1
    rho = I.tanh_slab(nx, ny, rl, rg, ny / 2.0)
    rho[solid == 1] = rg
    return solid, rho, rg, rl


def run(p, solid, rho, steps, wall_rho=None):
    s = O.OracleSim(p, solid=solid, wall_rho=wall_rho)
    s.init(rho)
    s.step(steps)
    return s


def test_uniform_field_equals_the_scalar_virtual_density():
    solid, rho, rg, rl = channel()
    p = cs_params(nx=8, ny=40, periodic_x=True, periodic_y=True, rho_s=0.3 * rl)
    a = run(p, solid, rho, 150)
    b = run(p, solid, rho, 150, wall_rho=np.full(solid.shape, 0.3 * rl))
    assert np.isfinite(a.get_state()).all()
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(a.fields()["rho"], b.fields()["rho"])


def test_mirror_symmetry_of_two_wall_densities():
    solid, rho, rg, rl = channel()
    ny = solid.shape[0]
    p = cs_params(nx=8, ny=ny, periodic_x=True, periodic_y=True, Fx=1e-6)
    lo, hi = rg, 0.3 * rl
    w_ab = np.where(np.arange(ny)[:, None] < ny // 2, lo, hi) * np.ones_like(solid, dtype=float)
    w_ba = w_ab[::-1]
    a = run(p, solid, rho, 300, wall_rho=w_ab)
    b = run(p, solid, rho[::-1], 300, wall_rho=w_ba)
    fa, fb = a.fields(), b.fields()
    assert np.abs(fa["rho"] - fb["rho"][::-1]).max() <= 1e-12 * rl
    assert np.abs(fa["ux"] - fb["ux"][::-1]).max() <= 1e-10 * np.abs(fa["ux"]).max()
    assert np.abs(fa["uy"] + fb["uy"][::-1]).max() <= 1e-10 * np.abs(fa["ux"]).max()
    # the field is used: the asymmetric channel differs from the uniform one
    c = run(p, solid, rho, 300, wall_rho=np.full(solid.shape, lo))
    assert np.abs(fa["rho"] - c.fields()["rho"]).max() > 1e-3 * rl


def test_liquid_like_wall_condenses_the_gas_next_to_it():
    solid, rho, rg, rl = channel()
    ny = solid.shape[0]
    p = cs_params(nx=8, ny=ny, periodic_x=True, periodic_y=True)
    w = np.where(np.arange(ny)[:, None] < ny // 2, rg, 0.3 * rl) * np.ones_like(solid, dtype=float)
    f = run(p, solid, rho, 400, wall_rho=w).fields()["rho"]
    below, above = f[1, 0], f[ny - 2, 0]  # first fluid rows next to the gas-like and liquid-like wall
    assert above > 3.0 * below, (below, above)
    assert abs(below - rg) < 0.2 * rg  # the gas-like wall leaves the gas near coexistence
    # and solid nodes report their own virtual density
    assert f[0, 0] == rg and f[ny - 1, 0] == 0.3 * rl


def test_annulus_with_a_gas_wetted_inner_and_liquid_wetted_outer_cylinder_is_stable():
    """The Sec. 3.2 configuration at quarter scale (R_i = 16, R_o = 64), van der Waals at
    T_r = 0.5, epsilon = 1.895: with one rho_s = rho_g the liquid against the outer cylinder
    detaches violently and the density leaves the range where psi is real within a few
    hundred steps; with the wall densities (rho_g inside, rho_l outside) it settles."""
    from tests.setups import vdw_case, vdw_params
    R_i, R_o = 16.0, 64.0
    n = 133
    c = (n - 1) / 2.0
    T, rg, rl = vdw_case(0.5)
    solid, _, q = I.annulus(n, n, R_i, R_o)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - c, y - c)
    w = np.where(r <= R_i, rg, rl)
    rho = 0.5 * (rl + rg) + 0.5 * (rl - rg) * np.tanh(2.0 * (r - (R_i + 0.25 * (R_o - R_i))) / 4.0)
    rho[solid == 1] = w[solid == 1]
    p = vdw_params(1.895, 0.5, nx=n, ny=n, periodic_x=True, periodic_y=True)
    f = run(p, solid, rho, 1500, wall_rho=w).fields()
    fl = solid == 0
    assert np.isfinite(f["rho"][fl]).all()
    assert np.hypot(f["ux"], f["uy"])[fl].max() < 0.02


def test_interpolated_walls_leak_mass_half_way_do_not():
    """The static two-phase annulus of the previous test: half-way links conserve the fluid
    mass to round-off; linear interpolated (Bouzidi) links, second order for the velocity,
    do not (measured 1.7e-4 relative in 2000 steps).  That leak made every long annulus run
    drift; the annular experiment therefore uses half-way links."""
    from tests.setups import vdw_case, vdw_params
    R_i, R_o, n = 16.0, 64.0, 133
    c = (n - 1) / 2.0
    T, rg, rl = vdw_case(0.5)
    solid, _, q = I.annulus(n, n, R_i, R_o)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - c, y - c)
    w = np.where(r <= R_i, rg, rl)
    rho = 0.5 * (rl + rg) + 0.5 * (rl - rg) * np.tanh(2.0 * (r - (R_i + 0.25 * (R_o - R_i))) / 4.0)
    rho[solid == 1] = w[solid == 1]
    p = vdw_params(1.895, 0.5, nx=n, ny=n, periodic_x=True, periodic_y=True)
    fl = solid == 0
    drift = {}
    for name, links in (("half-way", None), ("interpolated", q)):
        s = O.OracleSim(p, solid=solid, q=links, wall_rho=w)
        s.init(rho)
        s.step(500)
        m0 = s.fields()["rho"][fl].sum()
        s.step(2000)
        drift[name] = abs(s.fields()["rho"][fl].sum() - m0) / m0
    assert drift["half-way"] < 1e-12, drift
    assert drift["interpolated"] > 1e-5, drift
