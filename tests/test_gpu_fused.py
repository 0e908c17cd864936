"""The fused single-pass kernel against the two-pass kernel (bit-identical populations,
every storage precision, periodic and walled edges, partial strips and segments), and
against the FP64 oracle on sampled nodes at the full benchmark size."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_13407_gb300 import inputs as I
from paper_2604_13407_gb300 import lbm
from tests import gpu_cases as GC
from tests.setups import cs_case, cs_params

pytestmark = pytest.mark.gpu

PRECS = [(lbm.F64, {}), (lbm.F32, {}), (lbm.F16DEV, {}), (lbm.F16DEV, {"per_node_ref": 1}),
         (lbm.BF16DEV, {"per_node_ref": 1})]


def geometries():
    T, rg, rl = cs_case()
    g = {}
    p = cs_params(nx=256, ny=64, periodic_x=True, periodic_y=True, force_mode=1, Fy=-2e-5)
    g["periodic"] = GC.Case("periodic", p, I.droplet(256, 64, rl, rg, 12, 100.3, 30.2, periodic_x=True), 60)
    p = cs_params(nx=264, ny=37, periodic_x=True, periodic_y=False, Fx=2e-6)
    g["walls_y_ragged"] = GC.Case("walls_y_ragged", p, I.tanh_slab(264, 37, rl, rg, 15), 60)
    p = cs_params(nx=272, ny=96, periodic_x=False, periodic_y=True, force_mode=1, Fy=-1e-5)
    g["walls_x"] = GC.Case("walls_x", p, I.droplet(272, 96, rl, rg, 14, 135.6, 60.1, periodic_x=False), 60)
    return g


GEOMS = geometries()


def wall_geometries():
    """Fused-kernel sizes of the solid-wall cases: the 45-degree banded channel (solid bands
    where (x - y) mod 256 < 2, viscosity ratio 10) and the annulus with a resting inner and a
    moving outer cylinder through interpolated (Bouzidi) links."""
    T, rg, rl = cs_case()
    g = {}
    n = 256
    f = 1e-6
    p = cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True, Fx=f / 2 ** 0.5, Fy=f / 2 ** 0.5,
                  tau_l=1.0, tau_g=0.55, scheme=1)
    g["oblique256"] = GC.Case("oblique256", p, I.oblique_slab(n, rl, rg, 90), 400, solid=I.oblique_band_walls(n))
    solid, wall_u, q = I.annulus(n, n, 30.3, 118.6, u_wall_out=0.01)
    c0 = (n - 1) / 2
    r = np.hypot(np.arange(n)[None, :] - c0, np.arange(n)[:, None] - c0)
    ring = rg + 0.5 * (rl - rg) * (np.tanh(2 * (r - 55.0) / 4.0) - np.tanh(2 * (r - 88.0) / 4.0))
    p = cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True, scheme=1)
    g["annulus256"] = GC.Case("annulus256", p, np.where(solid == 1, rg, ring), 300, solid=solid, wall_u=wall_u, q=q)
    return g


WALL_GEOMS = wall_geometries()


@pytest.mark.parametrize("geom", sorted(WALL_GEOMS))
def test_fused_with_solid_walls_matches_oracle(geom):
    """One pass per step on solid-wall geometry (half-way, moving and interpolated links):
    the fused FP32 kernel against the FP64 oracle, every fluid node, 1e-4 of max |u| and of
    rho; FP64 contexts keep the two-pass kernels for such geometry."""
    c = WALL_GEOMS[geom]
    o = GC.run_oracle(c)
    g = GC.run_gpu(c, lbm.F32, lbm.KERNEL_FUSED)
    assert g.kernel_in_use == lbm.KERNEL_FUSED
    e_rho, e_u = GC.field_errors(g, o, c.solid)
    print("fused FP32 %s: e_u %.3e e_rho %.3e" % (geom, e_u, e_rho))
    assert e_u < 1e-4 and e_rho < 1e-4, (e_rho, e_u)
    assert GC.run_gpu(c, lbm.F64, lbm.KERNEL_AUTO, steps=1).kernel_in_use == lbm.KERNEL_TWO_PASS


@pytest.mark.parametrize("prec,kw", [(lbm.F32, {}), (lbm.F16DEV, {"per_node_ref": 1}), (lbm.BF16DEV, {"per_node_ref": 1})])
@pytest.mark.parametrize("geom", sorted(WALL_GEOMS))
def test_fused_with_solid_walls_equals_two_pass(geom, prec, kw):
    """The general-geometry fused kernel against the two-pass kernel on the fluid nodes
    (solid nodes hold no state), to the rounding of the packed arithmetic."""
    c = WALL_GEOMS[geom]
    a = GC.run_gpu(c, prec, lbm.KERNEL_TWO_PASS, steps=100, **kw)
    b = GC.run_gpu(c, prec, lbm.KERNEL_FUSED, steps=100, **kw)
    assert b.kernel_in_use == lbm.KERNEL_FUSED
    fluid = c.solid == 0
    A, B = a.get_state()[:, fluid], b.get_state()[:, fluid]
    tol = 1e-5 if prec == lbm.F32 else 2e-3
    assert np.all(np.isfinite(B))
    assert np.abs(A - B).max() < tol * np.abs(A).max(), np.abs(A - B).max() / np.abs(A).max()


@pytest.mark.parametrize("prec,kw", PRECS)
@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_fused_equals_two_pass(geom, prec, kw):
    """FP64 (compiled without multiply-add contraction): bit-identical.  The
    FP32-arithmetic kernels (FP32, FP16, BF16 storage) evaluate the one formulation of
    lbm_f32.cuh, per node in the two-pass kernel and on packed pairs in the fused kernel;
    the compiler fuses some packed multiply-add chains (a measured toolchain behaviour:
    the rounding of the pair instructions is not always the written one), so they agree
    to rounding; a staging or synchronisation fault would give O(1) differences."""
    c = GEOMS[geom]
    a = GC.run_gpu(c, prec, lbm.KERNEL_TWO_PASS, **kw)
    b = GC.run_gpu(c, prec, lbm.KERNEL_FUSED, **kw)
    assert a.kernel_in_use == lbm.KERNEL_TWO_PASS and b.kernel_in_use == lbm.KERNEL_FUSED
    A, B = a.get_state(), b.get_state()
    if prec == lbm.F64:
        assert np.array_equal(A, B)
        assert a.save_state() == b.save_state()
    else:
        tol = 1e-5 if prec == lbm.F32 else 2e-3
        assert np.all(np.isfinite(B))
        assert np.abs(A - B).max() < tol * np.abs(A).max(), np.abs(A - B).max() / np.abs(A).max()


@pytest.mark.parametrize("prec,kw", PRECS)
def test_fused_one_step_equals_two_pass(prec, kw):
    """From one shared state, one fused step and one two-pass step agree to a few ulps."""
    c = GEOMS["walls_y_ragged"]
    base = GC.run_gpu(c, prec, lbm.KERNEL_TWO_PASS, steps=25, **kw)
    A0 = base.get_state()
    out = []
    for kernel in (lbm.KERNEL_TWO_PASS, lbm.KERNEL_FUSED):
        s = lbm.Simulation(GC.gpu_params(c.params, prec, kernel, **kw))
        s.set_state(A0)
        s.step(1)
        out.append(s.get_state())
    tol = 0.0 if prec == lbm.F64 else (1e-6 if prec == lbm.F32 else 1e-3)
    assert np.abs(out[0] - out[1]).max() <= tol * np.abs(out[0]).max()


@pytest.mark.parametrize("geom", ["periodic", "walls_y_ragged", "walls_x"])
def test_fused_fp32_matches_oracle_whole_field(geom):
    """The kernel the benchmark times (fused, FP32) against the FP64 oracle over 600 steps,
    every node: max |du| <= 1e-4 max |u| and rho within 1e-4 relative."""
    c = GEOMS[geom]
    o = GC.run_oracle(c, steps=600)
    g = GC.run_gpu(c, lbm.F32, lbm.KERNEL_FUSED, steps=600)
    assert g.kernel_in_use == lbm.KERNEL_FUSED
    e_rho, e_u = GC.field_errors(g, o)
    print("fused FP32 %s 600 steps: e_u %.3e e_rho %.3e" % (geom, e_u, e_rho))
    assert e_u < 1e-4 and e_rho < 1e-4, (e_rho, e_u)


def test_fused_fp64_matches_oracle():
    c = GEOMS["walls_x"]
    o = GC.run_oracle(c)
    g = GC.run_gpu(c, lbm.F64, lbm.KERNEL_FUSED)
    assert g.kernel_in_use == lbm.KERNEL_FUSED
    e_rho, e_u = GC.field_errors(g, o)
    assert e_rho < 1e-10 and e_u < 1e-10, (e_rho, e_u)


def _patch(A, cx, cy, r=2):
    ny, nx = A.shape[1:]
    ys = [(cy + d) % ny for d in range(-r, r + 1)]
    xs = [(cx + d) % nx for d in range(-r, r + 1)]
    return A[:, ys][:, :, xs]


@pytest.mark.parametrize("prec,tol", [(lbm.F32, 2e-6), (lbm.F16DEV, 2e-3)])
def test_full_size_sampled_nodes_match_oracle(prec, tol):
    """8192 x 8192 periodic spinodal workload in the launch configuration bench.py times:
    the update of sampled nodes is recomputed by the oracle from the GPU's previous state
    (a 5 x 5 patch holds everything one node update depends on)."""
    import torch
    import bench
    n = 8192
    sim = bench.make_sim(n, prec)
    assert sim.kernel_in_use == lbm.KERNEL_FUSED
    sim.init_fields(bench.workload_rho(n))
    sim.step(3)
    before = torch.empty((9, n, n), dtype=torch.float64, device="cuda")
    sim.get_state(before)
    rng = np.random.default_rng(11)
    pts = [(0, 0), (n - 1, n - 1), (127, 4095), (128, 1), (n - 1, 0)] + [tuple(rng.integers(0, n, 2)) for _ in range(12)]
    patches = []
    for cx, cy in pts:
        ys = torch.tensor([(cy + d) % n for d in range(-2, 3)], device="cuda")
        xs = torch.tensor([(cx + d) % n for d in range(-2, 3)], device="cuda")
        patches.append(before.index_select(1, ys).index_select(2, xs).cpu().numpy())
    sim.step(1)
    sim.get_state(before)
    after = [before[:, cy, cx].cpu().numpy() for cx, cy in pts]
    del before
    p = O.Params(nx=5, ny=5, periodic_x=False, periodic_y=False, scheme=1, T=bench.T_07,
                 rho_l=bench.RHO_L, rho_g=bench.RHO_G, rho_s=bench.RHO_G, tau_l=bench.TAU, tau_g=bench.TAU)
    for P, a in zip(patches, after):
        s = O.OracleSim(p)
        s.set_state(P)
        s.step(1)
        ref = s.get_state()[:, 2, 2]
        assert np.abs(a - ref).max() < tol * np.abs(ref).max(), (a, ref)


@pytest.mark.parametrize("nx,ny,walls_x,geom,want", [
    (256, 256, False, None, lbm.KERNEL_TWO_PASS), (512, 512, False, None, lbm.KERNEL_FUSED),
    (2048, 2048, False, None, lbm.KERNEL_FUSED), (256, 2048, True, None, lbm.KERNEL_TWO_PASS),
    (512, 4096, True, None, lbm.KERNEL_FUSED), (256, 256, False, "band", lbm.KERNEL_TWO_PASS),
    (512, 512, False, "band", (lbm.KERNEL_TWO_PASS, lbm.KERNEL_FUSED)),
    (1024, 1024, False, "band", lbm.KERNEL_FUSED), (1024, 1024, False, "q", lbm.KERNEL_TWO_PASS)])
def test_auto_kernel_choice(nx, ny, walls_x, geom, want):
    """KERNEL_AUTO takes the one-pass kernel where it was measured faster: larger lattices,
    and solid or interpolated walls only on lattices large enough for the bulk to outweigh
    the walls' per-link work.  A pair (FP32, FP16) where the two storage types differ: the
    512^2 banded channel, where the two-pass kernels are faster in FP32 and slower in FP16."""
    for prec, w in zip((lbm.F32, lbm.F16DEV), want if isinstance(want, tuple) else (want, want)):
        p = lbm.default_params(nx=nx, ny=ny, periodic_x=0 if walls_x else 1, periodic_y=1, precision=prec,
                               per_node_ref=1, storage_scale_log2=18 if prec == lbm.F16DEV else 0)
        s = lbm.Simulation(p)
        if geom == "band":
            s.set_geometry(I.oblique_band_walls(nx))
        elif geom == "q":
            solid = np.zeros((ny, nx), np.uint8)
            solid[:, :2] = 1
            s.set_geometry(solid, None, np.full((8, ny, nx), 0.5))
        assert s.kernel_in_use == w, (nx, ny, geom, prec, s.kernel_in_use)
        s.close()
