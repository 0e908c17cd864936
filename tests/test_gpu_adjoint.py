"""GPU adjoint (lbm_adjoint_step, the transposed-step kernels) against the FP64 reference
adjoint of oracle/adjoint_ref.py and against central finite differences.

Tolerances.  FP64: J to 1e-11 relative plus 1e-15 absolute (J is a sum of O(1e-3) terms
that cancel by two orders of magnitude, or to zero for the y force on the walls of an
x-periodic channel), dJ/d(Fx, Fy, T) and lambda_0 to 1e-9 of their largest magnitude (the
GPU sums in another order than autograd).  FP32 arithmetic and storage: J to 1e-4
relative plus 1e-8 absolute, gradients and lambda_0 to 1e-5 of the largest magnitude (the
transposed step runs in FP32 about a forward state that carries FP32 rounding; measured
errors are below 2e-7 and 1e-6).  Finite differences at the full adjoint workload
(256 x 1024 channel, radius-20 droplet, 4000 steps, checkpoint every 200): central
differences with a step of 1e-4 relative in FP64; the FP64 and the FP32 adjoint gradients
within 1e-4 relative of them.

16-bit storage (FP16 and BF16 deviations, per-node reference density, stochastic
rounding): the transposed step runs in FP32 on the decoded states and takes the storage's
rounding as the identity.  Over one step the gradient therefore depends on the starting
state alone, which the storage holds exactly: against the FP64 reference adjoint at that
decoded state, 1e-5 as for FP32.  Over several steps the 16-bit trajectory leaves the FP64
one by the storage's rounding, and the gradient with it (bounds below)."""
import numpy as np
import pytest

from paper_2604_13407_gb300 import inputs as I
from paper_2604_13407_gb300 import lbm
from oracle import adjoint_ref as AR
from tests import gpu_cases as GC
from tests.setups import cs_case, cs_params
from tests.test_adjoint_ref import channel_case, droplet_case, initial_state

pytestmark = pytest.mark.gpu

OBJ = {"wall_force_y": lbm.OBJ_WALL_FORCE_Y, "mean_jx": lbm.OBJ_MEAN_JX}
PARAM_INDEX = (0, 1, 3)  # Fx, Fy, T; index 2 (G) is zero


def gpu_sim(p, solid, precision, A0, **kw):
    sim = lbm.Simulation(GC.gpu_params(p, precision, **kw))
    if solid is not None:
        sim.set_geometry(solid)
    sim.set_state(A0)
    return sim


@pytest.fixture(scope="module")
def references():
    out = {}
    for case in (channel_case, droplet_case):
        p, rho, solid = case()
        A0 = initial_state(p, rho, solid)
        for obj in OBJ:
            out[(case.__name__, obj)] = (p, solid, A0) + AR.objective_and_grad(p, A0, 12, obj, solid)
    return out


@pytest.mark.parametrize("case", ["channel_case", "droplet_case"])
@pytest.mark.parametrize("obj", sorted(OBJ))
@pytest.mark.parametrize("K", [1, 5, 12])
def test_fp64_adjoint_matches_reference(references, case, obj, K):
    p, solid, A0, J_ref, g_ref, lam_ref = references[(case, obj)]
    sim = gpu_sim(p, solid, lbm.F64, A0)
    J, g, lam = sim.adjoint(12, K, OBJ[obj], want_lambda0=True)
    assert abs(J - J_ref) <= 1e-11 * abs(J_ref) + 1e-15
    scale = np.abs(g_ref[list(PARAM_INDEX)]).max()
    for k in PARAM_INDEX:
        assert abs(g[k] - g_ref[k]) <= 1e-9 * scale, (k, g[k], g_ref[k])
    assert abs(g[2]) <= 1e-9 * scale
    assert np.abs(lam - lam_ref).max() <= 1e-9 * np.abs(lam_ref).max()
    assert sim.step_count == 12


@pytest.mark.parametrize("case", ["channel_case", "droplet_case"])
@pytest.mark.parametrize("obj", sorted(OBJ))
def test_fp32_adjoint_matches_reference(references, case, obj):
    p, solid, A0, J_ref, g_ref, lam_ref = references[(case, obj)]
    sim = gpu_sim(p, solid, lbm.F32, A0)
    J, g, lam = sim.adjoint(12, 4, OBJ[obj], want_lambda0=True)
    assert abs(J - J_ref) <= 1e-4 * abs(J_ref) + 1e-8
    scale = np.abs(g_ref[list(PARAM_INDEX)]).max()
    for k in PARAM_INDEX:
        assert abs(g[k] - g_ref[k]) <= 1e-5 * scale, (k, g[k], g_ref[k])
    assert abs(g[2]) <= 1e-5 * scale
    assert np.abs(lam - lam_ref).max() <= 1e-5 * np.abs(lam_ref).max()


def wide_droplet_case(nx=256, ny=40):
    """A droplet between walls at y = -1/2 and ny - 1/2, periodic in x, wide enough for the
    one-pass step kernel."""
    T, rg, rl = cs_case()
    p = cs_params(nx=nx, ny=ny, periodic_x=True, periodic_y=False, Fx=2e-6, Fy=-1e-6, scheme=1, tau_l=0.9,
                  tau_g=0.7)
    return p, I.droplet(nx, ny, rl, rg, 8.0, 0.4 * nx, 0.48 * ny, periodic_x=True, periodic_y=False)


@pytest.mark.parametrize("obj", sorted(OBJ))
def test_one_pass_recompute_matches_reference(obj):
    """A context that steps with the one-pass kernel recomputes each segment with it (the
    kernel also writing the psi field of the state it reads); one that steps with the
    two-pass kernels recomputes with those.  Both against the FP64 reference adjoint, at the
    FP32 tolerances."""
    p, rho = wide_droplet_case()
    A0 = initial_state(p, rho, None)
    J_ref, g_ref, lam_ref = AR.objective_and_grad(p, A0, 12, obj, None)
    scale = np.abs(g_ref[list(PARAM_INDEX)]).max()
    for kernel in (lbm.KERNEL_FUSED, lbm.KERNEL_TWO_PASS):
        sim = gpu_sim(p, None, lbm.F32, A0, kernel=kernel)
        assert sim.kernel_in_use == kernel
        J, g, lam = sim.adjoint(12, 5, OBJ[obj], want_lambda0=True)
        print("kernel %d: max |dg| / scale %.2e, lambda_0 %.2e" %
              (kernel, np.abs(g - g_ref)[list(PARAM_INDEX)].max() / scale,
               np.abs(lam - lam_ref).max() / np.abs(lam_ref).max()))
        assert abs(J - J_ref) <= 1e-4 * abs(J_ref) + 1e-8
        for k in PARAM_INDEX:
            assert abs(g[k] - g_ref[k]) <= 1e-5 * scale, (kernel, k, g[k], g_ref[k])
        assert np.abs(lam - lam_ref).max() <= 1e-5 * np.abs(lam_ref).max()


@pytest.mark.parametrize("obj", sorted(OBJ))
def test_replicated_lattice_adds_up(obj):
    """Four copies of a 512 x 1024 state side by side (2048 x 1024, periodic in x) evolve as
    four copies, so the mean x momentum and its gradient equal the single copy's and
    lambda_0 is a quarter of it per copy; the wall force, its gradient and lambda_0 add up
    over the copies (J four times the copy's, lambda_0 the copy's).  Both lattices step and
    recompute with the one-pass kernel; the larger one has four times the blocks, strips and
    per-block partial sums."""
    p1, rho = wide_droplet_case(512, 1024)
    p4, _ = wide_droplet_case(2048, 1024)
    small = lbm.Simulation(GC.gpu_params(p1, lbm.F32))
    small.init_fields(rho)
    A = small.get_state()
    small.set_state(A)
    big = lbm.Simulation(GC.gpu_params(p4, lbm.F32))
    big.set_state(np.tile(A, (1, 1, 4)))
    J1, g1, lam1 = small.adjoint(12, 5, OBJ[obj], want_lambda0=True)
    J4, g4, lam4 = big.adjoint(12, 5, OBJ[obj], want_lambda0=True)
    k = 1.0 if obj == "mean_jx" else 4.0
    scale = np.abs(g1[list(PARAM_INDEX)]).max()
    print("J %.9e / %.9e; max |dg| / scale %.2e" % (J1, J4 / k, np.abs(g4 / k - g1).max() / scale))
    assert abs(J4 / k - J1) <= 1e-6 * abs(J1)
    for q in PARAM_INDEX:
        assert abs(g4[q] / k - g1[q]) <= 1e-6 * scale, (q, g4[q], g1[q])
    lam_copy = lam4.reshape(9, 1024, 4, 512) * (4.0 if obj == "mean_jx" else 1.0)
    for c in range(4):
        assert np.abs(lam_copy[:, :, c, :] - lam1).max() <= 1e-6 * np.abs(lam1).max()


def test_checkpoint_interval_does_not_change_the_result(references):
    p, solid, A0, *_ = references[("droplet_case", "wall_force_y")]
    res = []
    for K in (1, 3, 12, 100):
        J, g, lam = gpu_sim(p, solid, lbm.F64, A0).adjoint(12, K, lbm.OBJ_WALL_FORCE_Y, want_lambda0=True)
        res.append((J, g, lam))
    for J, g, lam in res[1:]:
        # the gradients are summed in a fixed order; J includes one FP64 sum whose block
        # order is not fixed (the objective of the last state, added with atomics)
        assert abs(J - res[0][0]) <= 1e-14 * abs(res[0][0])
        assert np.abs(g - res[0][1]).max() <= 1e-13 * np.abs(res[0][1]).max()
        assert np.array_equal(lam, res[0][2])


def test_objective_only_and_state_after(references):
    """grad = lambda0 = NULL runs the forward sweep only; both calls leave the state of
    lbm_step(n)."""
    p, solid, A0, *_ = references[("droplet_case", "mean_jx")]
    a = gpu_sim(p, solid, lbm.F64, A0)
    J_full, _, _ = a.adjoint(12, 5, lbm.OBJ_MEAN_JX)
    b = gpu_sim(p, solid, lbm.F64, A0)
    J_only = b.objective(12, lbm.OBJ_MEAN_JX)
    c = gpu_sim(p, solid, lbm.F64, A0)
    c.step(12)
    assert abs(J_only - J_full) <= 1e-14 * abs(J_full)
    assert np.array_equal(a.get_state(), c.get_state())
    assert np.array_equal(b.get_state(), c.get_state())


def test_autograd_function_returns_the_adjoint_gradient(references):
    import torch
    p, solid, A0, J_ref, g_ref, _ = references[("channel_case", "mean_jx")]
    sim = gpu_sim(p, solid, lbm.F64, A0)
    snap = sim.save_state()
    theta = torch.tensor([p.Fx, p.Fy, p.G, p.T], dtype=torch.float64, requires_grad=True)
    J = lbm.time_averaged_objective(sim, theta, snap, 12, 4, lbm.OBJ_MEAN_JX)
    (3.0 * J).backward()
    assert abs(J.item() - J_ref) <= 1e-11 * abs(J_ref) + 1e-15
    g = theta.grad.numpy()
    scale = np.abs(g_ref[list(PARAM_INDEX)]).max()
    assert np.abs(g[[0, 1, 3]] - 3.0 * g_ref[[0, 1, 3]]).max() <= 3e-9 * scale


HALF = {"f16": lbm.F16DEV, "bf16": lbm.BF16DEV}
CASES = {"channel_case": channel_case, "droplet_case": droplet_case}


def half_sim(case, prec):
    p, rho, solid = CASES[case]()
    sim = gpu_sim(p, solid, HALF[prec], initial_state(p, rho, solid), per_node_ref=1)
    return p, solid, sim


@pytest.mark.parametrize("prec", sorted(HALF))
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("obj", sorted(OBJ))
def test_half_storage_one_step_is_the_transposed_step_at_the_stored_state(case, obj, prec):
    """n = 1: the gradient and lambda_0 against the FP64 reference adjoint at the stored
    (decoded) starting state to 1e-5 of their scale; J against the objective of the stored
    state after the step, read back in FP64: the library sums the same stored values after
    decoding each in FP32 (w_i rho_ref and the multiply-add, two roundings of 2^-24), so the
    two differ by at most 2^-22 sum |W_i| |A_i|."""
    p, solid, sim = half_sim(case, prec)
    A0 = sim.get_state()
    J_ref, g_ref, lam_ref = AR.objective_and_grad(p, A0, 1, obj, solid)
    J, g, lam = sim.adjoint(1, 1, OBJ[obj], want_lambda0=True)
    A1 = sim.get_state()
    J_stored = AR.objective_value(p, [A1], obj, solid)
    geo = AR.Geometry(p.nx, p.ny, bool(p.periodic_x), bool(p.periodic_y), solid)
    W_abs = np.abs(AR.weights(geo, obj).numpy()).reshape(A1.shape)
    scale = np.abs(g_ref[list(PARAM_INDEX)]).max()
    print("J %.9e (stored %.9e, unrounded step %.9e); max |dg| / scale %.2e" %
          (J, J_stored, J_ref, np.abs(g - g_ref)[list(PARAM_INDEX)].max() / scale))
    assert abs(J - J_stored) <= 2.0**-22 * (W_abs * np.abs(A1)).sum()
    for k in PARAM_INDEX:
        assert abs(g[k] - g_ref[k]) <= 1e-5 * scale, (k, g[k], g_ref[k])
    assert abs(g[2]) <= 1e-5 * scale
    assert np.abs(lam - lam_ref).max() <= 1e-5 * np.abs(lam_ref).max()


@pytest.mark.parametrize("prec", sorted(HALF))
def test_half_storage_recompute_repeats_the_forward_rounding(prec):
    """Checkpoints every step (no recompute) and one checkpoint for 12 steps (11 states
    recomputed, stochastically rounded with the forward steps' seeds) give the same
    gradient, lambda_0 and J: the recomputed 16-bit states are the forward ones bit for bit."""
    res = []
    for K in (1, 5, 12):
        _, _, sim = half_sim("droplet_case", prec)
        res.append(sim.adjoint(12, K, lbm.OBJ_WALL_FORCE_Y, want_lambda0=True))
    for J, g, lam in res[1:]:
        assert abs(J - res[0][0]) <= 1e-14 * abs(res[0][0])
        assert np.abs(g - res[0][1]).max() <= 1e-13 * np.abs(res[0][1]).max()
        assert np.array_equal(lam, res[0][2])


@pytest.mark.parametrize("prec,bound", [("f16", 5e-4), ("bf16", 3e-3)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_half_storage_twelve_steps_against_reference(references, case, prec, bound):
    """n = 12 from the same starting state as the FP64 reference adjoint: the 16-bit run
    follows its own rounded trajectory, so the gradient differs by the storage's rounding
    carried through the steps (measured: up to 6.7e-5 of the gradient's scale and 4.4e-5 of
    lambda_0's with FP16, 1.7e-4 and 2.7e-4 with BF16; the rounding is seeded by the step
    count, so runs repeat)."""
    for obj in sorted(OBJ):
        p, solid, A0, J_ref, g_ref, lam_ref = references[(case, obj)]
        sim = gpu_sim(p, solid, HALF[prec], A0, per_node_ref=1)
        J, g, lam = sim.adjoint(12, 4, OBJ[obj], want_lambda0=True)
        scale = np.abs(g_ref[list(PARAM_INDEX)]).max()
        err = np.abs(g - g_ref)[list(PARAM_INDEX)].max() / scale
        lerr = np.abs(lam - lam_ref).max() / np.abs(lam_ref).max()
        print("%s %s: max |dg| / scale %.2e, lambda_0 %.2e, J %.6e vs %.6e" % (case, obj, err, lerr, J, J_ref))
        assert err <= bound and lerr <= bound


def test_unsupported_combinations_are_rejected():
    T, rg, rl = cs_case()
    p = cs_params(nx=8, ny=8, periodic_x=True, periodic_y=True)
    sim = lbm.Simulation(GC.gpu_params(p, lbm.F64))
    sim.init_fields(np.full((8, 8), rl))
    solid = np.zeros((8, 8), np.uint8)
    solid[3, 3] = 1
    wall_u = np.zeros((2, 8, 8))
    wall_u[0, 3, 3] = 0.01
    sim.set_geometry(solid, wall_u)
    with pytest.raises(lbm.LbmError) as e:
        sim.adjoint(2, 1)
    assert e.value.status == 8
    sim.set_geometry(solid)
    with pytest.raises(lbm.LbmError) as e:
        sim.adjoint(0, 1)
    assert e.value.status == 1


def droplet_channel_params(precision, **kw):
    """The adjoint workload: 256 x 1024 channel, walls at x = -1/2 and 255.5, periodic in
    y, buoyant gravity g = 2e-6 downwards, improved scheme."""
    op = cs_params(nx=256, ny=1024, periodic_x=False, periodic_y=True, force_mode=1, Fx=0.0, Fy=-2e-6,
                   scheme=1, tau_l=0.8, tau_g=0.8)
    return op, GC.gpu_params(op, precision, **kw)


def droplet_channel_rho():
    T, rg, rl = cs_case()
    cx, cy = I.jittered_centre(4, 128.0, 900.0)
    return I.droplet(256, 1024, rl, rg, 20.0, cx, cy, periodic_x=False, periodic_y=True)


def test_full_workload_gradient_matches_central_differences():
    n, K = 4000, 200
    rho0 = droplet_channel_rho()
    op, p64 = droplet_channel_params(lbm.F64)

    def J_of(which=None, value=None, precision=lbm.F64):
        _, pp = droplet_channel_params(precision)
        sim = lbm.Simulation(pp)
        if which is not None:
            sim.set_param(which, value)
        sim.init_fields(rho0)
        return sim

    sim = J_of()
    J, g, _ = sim.adjoint(n, K, lbm.OBJ_WALL_FORCE_Y)
    checks = {}
    for which, name, base in ((lbm.PARAM_FY, "Fy", op.Fy), (lbm.PARAM_T, "T", op.T)):
        h = 1e-4 * abs(base)
        Jp = J_of(which, base + h).objective(n)
        Jm = J_of(which, base - h).objective(n)
        fd = (Jp - Jm) / (2 * h)
        checks[name] = (g[which], fd)
        print("d J/d %s: adjoint FP64 %.10e, central difference %.10e" % (name, g[which], fd))
        assert abs(g[which] - fd) <= 1e-4 * abs(fd), (name, g[which], fd)
    # G drops out of the step: the normalised sensitivity G dJ/dG vanishes
    assert abs(g[2] * op.G) <= 1e-8 * abs(g[3] * op.T)
    # FP32 transposed step on the FP32 forward run
    sim32 = J_of(precision=lbm.F32)
    J32, g32, _ = sim32.adjoint(n, K, lbm.OBJ_WALL_FORCE_Y)
    for which, name in ((lbm.PARAM_FY, "Fy"), (lbm.PARAM_T, "T")):
        fd = checks[name][1]
        print("d J/d %s: adjoint FP32 %.10e" % (name, g32[which]))
        assert abs(g32[which] - fd) <= 1e-4 * abs(fd), (name, g32[which], fd)
    # FP16 storage (per-node reference, stochastic rounding): the transposed step of the
    # 16-bit run; its trajectory differs from the FP32 one by the storage's rounding
    # (measured: 2.1e-5 of the central difference for Fy, 1.9e-4 for T)
    _, p16 = droplet_channel_params(lbm.F16DEV, per_node_ref=1, storage_scale_log2=18)
    sim16 = lbm.Simulation(p16)
    sim16.init_fields(rho0)
    J16, g16, _ = sim16.adjoint(n, K, lbm.OBJ_WALL_FORCE_Y)
    print("J: FP64 %.10e, FP32 %.10e, FP16 storage %.10e" % (J, J32, J16))
    for which, name in ((lbm.PARAM_FY, "Fy"), (lbm.PARAM_T, "T")):
        fd = checks[name][1]
        print("d J/d %s: adjoint with FP16 storage %.10e (%.2e of the central difference)" %
              (name, g16[which], abs(g16[which] - fd) / abs(fd)))
        assert abs(g16[which] - fd) <= 2e-3 * abs(fd), (name, g16[which], fd)
