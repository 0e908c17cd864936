"""GPU parity: the CUDA library through the C ABI against the FP64 oracle on the same
seeded inputs.

Tolerances.  FP64: 1e-10 relative on rho and on u (max |du| / max |u|); the FP64 path
evaluates the formulas in plain order, so it is in fact bit-identical.  FP32: 1e-4 of
max |u| and 1e-4 relative on rho.  FP16/BF16 deviation storage with a per-node
reference density: the 11-bit (FP16) or 8-bit (BF16) significand of the stored deviation
bounds the velocity error near interfaces, where the populations of the light phase carry
the large pairwise force; measured errors are ~5e-3 (FP16) and ~1e-1 (BF16) of max |u|,
so the bounds below are 2e-2 and 3e-1."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_13407_gb300 import lbm
from tests import gpu_cases as GC

pytestmark = pytest.mark.gpu

CASES = GC.cases()


@pytest.fixture(scope="module")
def oracle_runs():
    return {name: GC.run_oracle(c) for name, c in CASES.items()}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_two_pass_matches_oracle(name, oracle_runs):
    c = CASES[name]
    sim = GC.run_gpu(c, lbm.F64, lbm.KERNEL_TWO_PASS)
    e_rho, e_u = GC.field_errors(sim, oracle_runs[name], c.solid)
    assert e_rho < 1e-10 and e_u < 1e-10, (e_rho, e_u)


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_auto_kernel_matches_oracle(name, oracle_runs):
    c = CASES[name]
    sim = GC.run_gpu(c, lbm.F64, lbm.KERNEL_AUTO)
    e_rho, e_u = GC.field_errors(sim, oracle_runs[name], c.solid)
    assert e_rho < 1e-10 and e_u < 1e-10, (e_rho, e_u, sim.kernel_in_use)


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_matches_oracle(name, oracle_runs):
    c = CASES[name]
    sim = GC.run_gpu(c, lbm.F32)
    e_rho, e_u = GC.field_errors(sim, oracle_runs[name], c.solid)
    assert e_u < 1e-4 and e_rho < 1e-4, (e_rho, e_u)


HALF_TOL = {lbm.F16DEV: 2e-2, lbm.BF16DEV: 3e-1}


@pytest.mark.parametrize("prec", [lbm.F16DEV, lbm.BF16DEV])
@pytest.mark.parametrize("name", ["droplet", "channel_s1", "annulus"])
def test_half_storage_per_node_ref_matches_oracle(name, prec, oracle_runs):
    c = CASES[name]
    sim = GC.run_gpu(c, prec, per_node_ref=1)
    e_rho, e_u = GC.field_errors(sim, oracle_runs[name], c.solid)
    assert e_u < HALF_TOL[prec] and e_rho < HALF_TOL[prec], (e_rho, e_u)


def test_one_step_from_oracle_state_fp64():
    c = CASES["annulus"]
    o = GC.run_oracle(c, steps=37)
    A0 = o.get_state()
    sim = lbm.Simulation(GC.gpu_params(c.params, lbm.F64))
    sim.set_geometry(c.solid, c.wall_u, c.q, c.fext)
    sim.set_state(A0)
    assert np.array_equal(sim.get_state()[:, c.solid == 0], A0[:, c.solid == 0])
    sim.step(1)
    o.step(1)
    fluid = c.solid == 0
    d = np.abs(sim.get_state() - o.get_state())[:, fluid]
    assert d.max() < 1e-15


@pytest.mark.parametrize("name", ["annulus", "channel_s1", "droplet"])
def test_diagnostics_match_oracle(name, oracle_runs):
    c = CASES[name]
    sim = GC.run_gpu(c, lbm.F64)
    dg = sim.diagnostics()
    do = oracle_runs[name].diagnostics()
    scale = np.array([do[0], do[0], do[0], abs(do[3]) + abs(do[4]) + 1e-30, abs(do[3]) + abs(do[4]) + 1e-30,
                      abs(do[5]) + abs(do[6]) + 1e-30, abs(do[5]) + abs(do[6]) + 1e-30,
                      do[8] * do[9] + 1e-30, do[8] + 1e-30, do[9]])
    err = np.abs(dg - do) / scale
    assert err[[0, 8, 9]].max() < 1e-10, (dg, do)
    assert err[[1, 2, 3, 4, 5, 6, 7]].max() < 1e-7, (dg, do)


def test_c1_full_run_both_schemes():
    """The 4 x 128 grid-aligned two-phase Poiseuille case, 20k steps, FP64, both schemes."""
    from tests.setups import cs_case, cs_params
    from paper_2604_13407_gb300 import inputs as I
    T, rg, rl = cs_case()
    for scheme in (0, 1):
        p = cs_params(nx=4, ny=128, periodic_x=True, periodic_y=False, Fx=1e-7, scheme=scheme)
        case = GC.Case("c1", p, I.tanh_slab(4, 128, rl, rg, 64), 20000)
        o = GC.run_oracle(case)
        g = GC.run_gpu(case, lbm.F64)
        e_rho, e_u = GC.field_errors(g, o)
        assert e_rho < 1e-10 and e_u < 1e-10, (scheme, e_rho, e_u)
        g32 = GC.run_gpu(case, lbm.F32)
        e_rho, e_u = GC.field_errors(g32, o)
        assert e_u < 1e-4, (scheme, e_rho, e_u)


def test_save_load_roundtrip_bitwise():
    c = CASES["droplet"]
    for prec, kw in ((lbm.F32, {}), (lbm.F16DEV, {"per_node_ref": 1}), (lbm.F64, {})):
        sim = GC.run_gpu(c, prec, steps=20, **kw)
        blob = sim.save_state()
        sim.step(15)
        after = sim.get_state()
        sim.load_state(blob)
        sim.step(15)
        assert np.array_equal(sim.get_state(), after)


def test_nan_is_reported():
    c = CASES["droplet"]
    sim = GC.run_gpu(c, lbm.F32, steps=1)
    A = sim.get_state()
    A[3, 5, 7] = np.nan
    sim.set_state(A)
    sim.step(2)
    with pytest.raises(lbm.LbmError) as e:
        sim.diagnostics()
    assert e.value.status == 5
