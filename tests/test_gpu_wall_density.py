"""GPU parity of the per-node virtual wall density (lbm_set_wall_density) against the FP64
oracle (or_set_wall_density), through the C ABI.

Tolerances as in test_gpu_parity.py: FP64 bit-identical (the FP64 path evaluates in the
oracle's order; checked to 1e-12), FP32 1e-4 of max |u| and 1e-3 relative on rho.  Cases:
the channel with a gas-like wall below and a liquid-like wall above (Carnahan-Starling,
driven along the walls), and a small annulus with interpolated bounce-back, a gas-wetted
inner and a liquid-wetted outer cylinder (van der Waals at T_r = 0.5, epsilon = 1.895, the
Sec. 3.2 set-up at one eighth of its size)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_13407_gb300 import inputs as I
from paper_2604_13407_gb300 import lbm
from tests import gpu_cases as GC
from tests.setups import cs_case, cs_params, vdw_case, vdw_params
from tests.test_wall_density import channel

pytestmark = pytest.mark.gpu


def channel_case():
    solid, rho, rg, rl = channel()
    ny = solid.shape[0]
    p = cs_params(nx=8, ny=ny, periodic_x=True, periodic_y=True, Fx=1e-6)
    w = np.where(np.arange(ny)[:, None] < ny // 2, rg, 0.3 * rl) * np.ones_like(solid, dtype=float)
    return p, solid, None, w, rho, 300


def annulus_case():
    R_i, R_o, n = 8.0, 32.0, 69
    c = (n - 1) / 2.0
    T, rg, rl = vdw_case(0.5)
    solid, _, q = I.annulus(n, n, R_i, R_o)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - c, y - c)
    w = np.where(r <= R_i, rg, rl)
    rho = 0.5 * (rl + rg) + 0.5 * (rl - rg) * np.tanh(2.0 * (r - (R_i + 0.25 * (R_o - R_i))) / 4.0)
    rho[solid == 1] = w[solid == 1]
    p = vdw_params(1.895, 0.5, nx=n, ny=n, periodic_x=True, periodic_y=True, scheme=1)
    return p, solid, q, w, rho, 400


CASES = {"channel": channel_case, "annulus": annulus_case}


def gpu_run(case, precision, wall=True):
    p, solid, q, w, rho, steps = case
    gp = GC.gpu_params(p, precision)
    if p.eos == 0:
        gp.rho_max = 9.0  # van der Waals psi is real up to about 9.9 at T_r = 0.5
    sim = lbm.Simulation(gp)
    sim.set_geometry(solid, None, q)
    if wall:
        sim.set_wall_density(w)
    sim.init_fields(rho)
    sim.step(steps)
    return sim


def oracle_run(case):
    p, solid, q, w, rho, steps = case
    s = O.OracleSim(p, solid=solid, q=q, wall_rho=w)
    s.init(rho)
    s.step(steps)
    return s


@pytest.fixture(scope="module")
def runs():
    return {name: (make(), oracle_run(make())) for name, make in CASES.items()}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_matches_oracle(runs, name):
    case, ref = runs[name]
    sim = gpu_run(case, lbm.F64)
    rg, ug, vg = sim.moments()
    f = ref.fields()
    fluid = case[1] == 0
    umax = max(np.abs(f["ux"][fluid]).max(), np.abs(f["uy"][fluid]).max())
    assert np.isfinite(rg).all()
    assert np.abs(rg - f["rho"]).max() <= 1e-12 * f["rho"].max()
    assert max(np.abs(ug - f["ux"]).max(), np.abs(vg - f["uy"]).max()) <= 1e-12 * umax
    # solid nodes report their own virtual density
    assert np.array_equal(rg[case[1] == 1], case[3][case[1] == 1])


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_matches_oracle(runs, name):
    case, ref = runs[name]
    sim = gpu_run(case, lbm.F32)
    rg, ug, vg = sim.moments()
    f = ref.fields()
    fluid = case[1] == 0
    umax = max(np.abs(f["ux"][fluid]).max(), np.abs(f["uy"][fluid]).max(), 1e-3)
    du = max(np.abs(ug - f["ux"])[fluid].max(), np.abs(vg - f["uy"])[fluid].max())
    assert du < 1e-4 * umax
    assert np.max(np.abs(rg - f["rho"])[fluid] / f["rho"][fluid]) < 1e-3


@pytest.mark.parametrize("precision", [lbm.F64, lbm.F32])
def test_uniform_field_equals_scalar_walls(precision):
    p, solid, q, w, rho, steps = channel_case()
    a = gpu_run((p, solid, q, np.full(solid.shape, p.rho_s), rho, steps), precision)
    b = gpu_run((p, solid, q, None, rho, steps), precision, wall=False)
    assert np.array_equal(a.get_state(), b.get_state())


def test_invalid_wall_density_is_rejected_and_adjoint_refuses_the_field():
    p, solid, q, w, rho, steps = channel_case()
    sim = lbm.Simulation(GC.gpu_params(p, lbm.F64))
    sim.set_geometry(solid)
    bad = w.copy()
    bad[0, 0] = -1.0
    with pytest.raises(lbm.LbmError) as e:
        sim.set_wall_density(bad)
    assert e.value.status == 1
    sim.set_wall_density(w)
    sim.init_fields(rho)
    with pytest.raises(lbm.LbmError) as e:
        sim.adjoint(2, 1)
    assert e.value.status == 8
    sim.set_wall_density(None)
    sim.init_fields(rho)
    J = sim.objective(2)
    assert np.isfinite(J)
