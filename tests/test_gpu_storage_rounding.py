"""Stochastic rounding of the 16-bit deviation storage (lbm_params.storage_rounding = 1).

Rounding to nearest makes the same error at every node of a region whose state is uniform
to better than the storage's precision, and the collision hands the node the same state
again the next step, so the errors add up: a uniformly translating fluid gains or loses
mass and momentum at a steady rate.  Stochastic rounding rounds up with probability equal
to the discarded fraction of an ulp, so each stored value is exact in expectation and the
errors of different nodes and steps are independent: the same fluid keeps its mass and
momentum to a random walk.  The random bits hash the node pair, population and step, so
both step kernels round every value alike and a run repeats exactly."""
import numpy as np
import pytest

from paper_2604_13407_gb300 import lbm
from tests import gpu_cases as GC
from tests.setups import cs_case, cs_params

pytestmark = pytest.mark.gpu

HALF = [(lbm.F16DEV, 18), (lbm.BF16DEV, 0)]


def _translating(prec, scale, rounding, kernel=lbm.KERNEL_AUTO, n=256, u=(0.05, 0.02)):
    """A uniform liquid (rho_l of the Carnahan-Starling EOS at 0.7 T_c) moving at u on a
    periodic n x n lattice: no force acts and the exact update keeps the state."""
    T, rg, rl = cs_case()
    p = GC.gpu_params(cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True), prec, kernel, per_node_ref=1,
                      storage_rounding=rounding)
    p.storage_scale_log2 = scale
    s = lbm.Simulation(p)
    s.init_fields(np.full((n, n), rl), np.full((n, n), u[0]), np.full((n, n), u[1]))
    return s


def _ulp(prec, x, scale):
    """Spacing of the storage type at |x| 2^scale, in units of x."""
    e = np.floor(np.log2(abs(x) * 2.0 ** scale))
    return 2.0 ** (e - (10 if prec == lbm.F16DEV else 7) - scale)


@pytest.mark.parametrize("prec,scale", HALF)
def test_uniform_translation_keeps_mass_and_momentum(prec, scale):
    """2000 steps of the uniformly translating liquid.  Stochastic rounding: every stored
    value is off by a zero-mean error of at most an ulp of the largest deviation (standard
    deviation at most half an ulp), independent between nodes and steps, so the mass and
    each momentum component take a random walk of at most 3/2 ulp sqrt(nodes x steps);
    the drift stays within 5 of those.  Rounding to nearest repeats one error at every node
    and step: its mass drift is many times larger."""
    n, steps, u = 256, 2000, (0.05, 0.02)
    T, rg, rl = cs_case()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    eu = ex * u[0] + ey * u[1]
    dev = w * rl * (3 * eu + 4.5 * eu * eu - 1.5 * (u[0] ** 2 + u[1] ** 2))
    walk = 5 * 1.5 * _ulp(prec, np.abs(dev).max(), scale) * np.sqrt(n * n * steps)
    drift = {}
    for rounding in (0, 1):
        s = _translating(prec, scale, rounding, n=n, u=u)
        d0 = s.diagnostics()
        s.step(steps)
        d1 = s.diagnostics()
        drift[rounding] = tuple(abs(d1[q] - d0[q]) for q in range(3))
        s.close()
    print("mass, jx, jy drift: nearest %s, stochastic %s, random-walk bound %.3g" % (drift[0], drift[1], walk))
    assert max(drift[1]) < walk, drift
    assert drift[1][0] * 10 < drift[0][0], drift


@pytest.mark.parametrize("prec,scale", HALF)
def test_both_kernels_round_alike(prec, scale):
    """One step of the same droplet state (40 steps old) by the two-pass and by the fused
    kernel.  Their FP32 arithmetic agrees to rounding, not bit for bit: where the density
    differs in its last bit, the deviation f - w_i rho differs by an ulp of w_i rho, a
    sizeable fraction of the deviation's own ulp, and the stored values can round apart.
    With rounding to nearest that happens to a few percent of the values; stochastic
    rounding with the same random bits in both kernels does no worse (with independent
    bits about a third of the changed values would differ)."""
    T, rg, rl = cs_case()
    n = 256
    from paper_2604_13407_gb300 import inputs as I
    p0 = cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True, scheme=1)
    rho0 = I.droplet(n, n, rl, rg, 40, 127.3, 121.6, periodic_x=True)

    def sim(kernel, rounding):
        p = GC.gpu_params(p0, prec, kernel, per_node_ref=1, storage_rounding=rounding)
        p.storage_scale_log2 = scale
        return lbm.Simulation(p)

    s0 = sim(lbm.KERNEL_TWO_PASS, 1)
    s0.init_fields(rho0)
    s0.step(40)
    A0 = s0.get_state()
    s0.close()
    frac = {}
    for rounding in (0, 1):
        states = {}
        for kernel in (lbm.KERNEL_TWO_PASS, lbm.KERNEL_FUSED):
            s = sim(kernel, rounding)
            s.set_state(A0)
            s.step(1)
            assert s.kernel_in_use == kernel and s.step_count == 1
            states[kernel] = s.get_state()
            s.close()
        a, b = states[lbm.KERNEL_TWO_PASS], states[lbm.KERNEL_FUSED]
        frac[rounding] = (np.mean(a != A0), np.mean(a != b))
    print("changed by the step / differing between the kernels: nearest %s, stochastic %s" % (frac[0], frac[1]))
    assert frac[1][0] > 0.2
    assert frac[1][1] < 2 * frac[0][1] + 1e-3, frac


@pytest.mark.parametrize("prec,scale", HALF)
def test_stochastic_rounding_repeats(prec, scale):
    """The random bits depend only on the node, population and step: two runs agree bit
    for bit, and a saved state resumes bit for bit."""
    runs = []
    for _ in range(2):
        s = _translating(prec, scale, 1, n=64)
        s.step(50)
        runs.append(s.get_state())
        blob = s.save_state()
        s.step(20)
        after = s.get_state()
        s.load_state(blob)
        s.step(20)
        assert np.array_equal(s.get_state(), after)
        s.close()
    assert np.array_equal(runs[0], runs[1])


def test_channel_accuracy_with_stochastic_rounding(oracle_channel):
    """The 4 x 64 two-phase channel (3000 steps) in FP16 with per-node reference and
    stochastic rounding against the FP64 oracle, beside rounding to nearest.  The random
    rounding breaks the channel's mirror symmetry, which lets the liquid slab start to
    translate between the walls (the unstable mode of this set-up), so the density error is
    bounded loosely."""
    c, o = oracle_channel
    errs = {}
    for rounding in (0, 1):
        sim = GC.run_gpu(c, lbm.F16DEV, per_node_ref=1, storage_rounding=rounding)
        e_rho, e_u = GC.field_errors(sim, o, c.solid)
        errs[rounding] = (e_u, e_rho)
        sim.close()
    print("FP16 channel e_u, e_rho: nearest %s, stochastic %s" % (errs[0], errs[1]))
    assert errs[1][0] < 5e-2 and errs[1][1] < 0.5, errs


@pytest.fixture(scope="module")
def oracle_channel():
    c = GC.cases()["channel_s1"]
    return c, GC.run_oracle(c)
