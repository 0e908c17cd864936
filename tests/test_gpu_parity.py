"""GPU parity: the CUDA library through the C ABI against the FP64 oracle on the same
seeded inputs.

Tolerances.  FP64: 1e-10 relative on rho and on u (max |du| / max |u|); the FP64 path
evaluates the formulas in plain order, so it is in fact bit-identical.  FP32: 1e-4 of
max |u| and 1e-4 relative on rho, on every case including the 20k-step grid-aligned
channel.  FP16/BF16 deviation storage with a per-node reference density: the 11-bit
(FP16) or 8-bit (BF16) significand of the stored deviation bounds the velocity error near
interfaces, where the populations of the light phase carry the large pairwise force;
measured errors are ~5e-3 (FP16) and ~1e-1 (BF16) of max |u|, so the bounds below are
2e-2 and 5e-1."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_13407_gb300 import inputs as I
from paper_2604_13407_gb300 import lbm
from tests import gpu_cases as GC
from tests.setups import cs_case, cs_params

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
    """FP32: max |du| <= 1e-4 max(max |u|, 1e-3) (FP32 resolves u to ~1e-8 absolute at
    these densities, so a near-static case is compared against 1e-3) and rho within 1e-4."""
    c = CASES[name]
    sim = GC.run_gpu(c, lbm.F32)
    rg, ug, vg = sim.moments()
    ro, uo, vo = oracle_runs[name].moments()
    fluid = np.ones_like(ro, dtype=bool) if c.solid is None else c.solid == 0
    umax = max(np.abs(uo[fluid]).max(), np.abs(vo[fluid]).max(), 1e-3)
    du = max(np.abs(ug - uo)[fluid].max(), np.abs(vg - vo)[fluid].max())
    e_rho = np.max(np.abs(rg - ro)[fluid] / ro[fluid])
    assert du < 1e-4 * umax and e_rho < 1e-4, (e_rho, du / umax)


HALF_TOL = {lbm.F16DEV: (2e-2, 5e-2), lbm.BF16DEV: (5e-1, 1.0)}


@pytest.mark.parametrize("prec", [lbm.F16DEV, lbm.BF16DEV])
@pytest.mark.parametrize("name", ["droplet", "channel_s1", "annulus"])
def test_half_storage_per_node_ref_matches_oracle(name, prec, oracle_runs):
    """Whole-run error of deviation storage (stochastic rounding, the default; measured on
    the channel: FP16 3e-3 of max |u|, BF16 ~1e-1); the bounds catch codec faults, the
    one-step test below pins the rounding."""
    c = CASES[name]
    sim = GC.run_gpu(c, prec, per_node_ref=1)
    e_rho, e_u = GC.field_errors(sim, oracle_runs[name], c.solid)
    tu, tr = HALF_TOL[prec]
    assert e_u < tu and e_rho < tr, (e_rho, e_u)


@pytest.mark.parametrize("prec,bits", [(lbm.F16DEV, 11), (lbm.BF16DEV, 8)])
@pytest.mark.parametrize("per_node", [0, 1])
@pytest.mark.parametrize("rounding", [0, 1])
def test_half_storage_one_step_is_rounded_deviation(prec, bits, per_node, rounding):
    """One step from a state the codec represents exactly: every stored population differs
    from the oracle's FP64 update by at most the rounding error of its deviation -- half an
    ulp (2^-bits relative) rounded to nearest, less than one ulp (2^(1-bits)) rounded
    stochastically -- plus FP32 arithmetic (1e-6 of the population)."""
    c = CASES["droplet"]
    o = GC.run_oracle(c, steps=30)
    sim = lbm.Simulation(GC.gpu_params(c.params, prec, per_node_ref=per_node, storage_rounding=rounding))
    sim.set_state(o.get_state())
    A0 = sim.get_state()          # decoded: exactly representable
    o.set_state(A0)
    sim.step(1)
    o.step(1)
    got, ref = sim.get_state(), o.get_state()
    if per_node:
        rho_ref = ref.sum(axis=0)[None]
    else:
        rho_ref = c.params.rho_g
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    dev = np.abs(ref - w * rho_ref)
    bound = dev * 2.0 ** (-bits + rounding) * 1.01 + 1e-6 * np.abs(ref) + 1e-12
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


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
    """FP64 diagnostics against the oracle's.  Sums that cancel by symmetry (total force,
    wall momentum) are compared absolutely against the mass scale."""
    c = CASES[name]
    sim = GC.run_gpu(c, lbm.F64)
    dg = sim.diagnostics()
    do = oracle_runs[name].diagnostics()
    assert abs(dg[0] - do[0]) < 1e-12 * do[0]
    assert abs(dg[8] - do[8]) < 1e-12 * do[0]
    assert abs(dg[9] - do[9]) < 1e-10 * do[9]
    assert np.abs(dg[1:8] - do[1:8]).max() < 1e-12 * do[0], (dg, do)


def test_fp32_diagnostics_sum_the_fp32_state_exactly():
    """FP32 storage: the diagnostics add the per-node FP32 densities of the kernel (pulled
    populations summed in the kernel's order) with compensated per-thread sums and FP64
    across threads, so the mass equals the exact sum of those FP32 densities to ~1e-14."""
    import math
    c = CASES["droplet"]  # periodic in x and y: the pull is a permutation
    sim = GC.run_gpu(c, lbm.F32, steps=30)
    A = sim.get_state().astype(np.float32)
    f = [np.roll(np.roll(A[i], lbm_ey(i), axis=0), lbm_ex(i), axis=1) for i in range(9)]
    # the kernel's density: deviations d_i = f_i - (w_i/w_0) f_0 (exact), pairwise sums,
    # rho = (9/4) f_0 + (s14 + s58) with one rounding (a multiply-add)
    q0, o0 = f[0] * np.float32(0.25), f[0] * np.float32(0.0625)
    d = [f[0]] + [f[i] - q0 for i in (1, 2, 3, 4)] + [f[i] - o0 for i in (5, 6, 7, 8)]
    s14 = (d[1] + d[3]) + (d[2] + d[4])
    s58 = (d[5] + d[7]) + (d[6] + d[8])
    rho = (2.25 * f[0].astype(np.float64) + (s14 + s58).astype(np.float64)).astype(np.float32)
    assert rho.dtype == np.float32
    exact = math.fsum(rho.astype(np.float64).ravel())
    d = sim.diagnostics()
    assert abs(d[0] - exact) <= 1e-14 * exact, (d[0], exact)


def lbm_ex(i):
    return [0, 1, 0, -1, 0, 1, -1, -1, 1][i]


def lbm_ey(i):
    return [0, 0, 1, 0, -1, 1, 1, -1, -1][i]


def test_wall_momentum_balance_on_gpu():
    """Exact discrete balance of the streaming (as pinned for the oracle):
    sum j(n+1) = sum j(n) + sum F(n) - D(n+1)."""
    c = CASES["channel_s1"]
    sim = GC.run_gpu(c, lbm.F64, steps=40)
    for _ in range(3):
        d0 = sim.diagnostics()
        sim.step(1)
        d1 = sim.diagnostics()
        for k in range(2):
            assert abs(d1[1 + k] - (d0[1 + k] + d0[3 + k] - d1[5 + k])) < 1e-13 * d0[0]


def test_c1_full_run_both_schemes():
    """The 4 x 128 grid-aligned two-phase Poiseuille case, 20k steps, both schemes.
    FP64 is compared at 1e-10 (it is bit-identical), FP32 at 1e-4 of max |u| after 3000
    and after 20000 steps, and at 1e-4 relative on rho after 3000 steps.  At 20k steps the
    FP32 density keeps ~1e-4 relative near the interfaces: a net mass drift of ~3e-10 per
    step (the rounding of the nine stored populations; each node's mass is closed, but not
    exactly) moves the interfaces by ~1e-4 node; the bound there is 5e-4."""
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
        print("C1 FP32 20k steps scheme %d: e_u %.3e e_rho %.3e" % (scheme, e_u, e_rho))
        assert e_u < 1e-4 and e_rho < 5e-4, (scheme, e_rho, e_u)
        o3 = GC.run_oracle(case, steps=3000)
        g3 = GC.run_gpu(case, lbm.F32, steps=3000)
        e_rho, e_u = GC.field_errors(g3, o3)
        print("C1 FP32 3000 steps scheme %d: e_u %.3e e_rho %.3e" % (scheme, e_u, e_rho))
        assert e_u < 1e-4 and e_rho < 1e-4, (scheme, e_rho, e_u)


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


def test_moments_into_host_buffers():
    """moments(out=...) with numpy arrays or (pinned) torch CPU tensors gives the same values
    as the arrays it allocates itself."""
    import torch
    c = CASES["droplet"]
    sim = GC.run_gpu(c, lbm.F32, steps=10)
    ref = sim.moments()
    n = sim.n
    for bufs in ([np.empty(n) for _ in range(3)], [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(3)]):
        got = sim.moments(out=bufs)
        for a, b in zip(got, ref):
            a = a.numpy() if hasattr(a, "numpy") else a
            assert np.array_equal(a.reshape(b.shape), b)
    with pytest.raises(ValueError):
        sim.moments(out=[np.empty(n, dtype=np.float32) for _ in range(3)])


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


@pytest.mark.parametrize("kernel", [lbm.KERNEL_TWO_PASS, lbm.KERNEL_FUSED])
def test_diag_every_stops_at_the_first_check(kernel):
    """diag_every = 10: lbm_step waits at step counts 10, 20, ...; a state that turns
    non-finite stops the call at the first such count with LBM_ENAN.  A healthy state runs
    through every check; diag_every = 0 never checks."""
    n = 256
    T, rg, rl = cs_case()
    p0 = cs_params(nx=n, ny=48, periodic_x=True, periodic_y=False, scheme=1)
    rho0 = I.droplet(n, 48, rl, rg, 10.0, 100.3, 23.6, periodic_x=True, periodic_y=False)
    for every in (10, 0):
        sim = lbm.Simulation(GC.gpu_params(p0, lbm.F32, kernel, diag_every=every))
        assert sim.kernel_in_use == kernel
        sim.init_fields(rho0)
        sim.step(35)
        assert sim.step_count == 35
        sim.step(3)
        A = sim.get_state()
        A[3, 20, 7] = np.nan
        sim.set_state(A)  # resets the step count
        if every:
            with pytest.raises(lbm.LbmError) as e:
                sim.step(100)
            assert e.value.status == 5 and sim.step_count == 10
        else:
            sim.step(100)
            assert sim.step_count == 100
        sim.close()
