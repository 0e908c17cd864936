"""The FP32-arithmetic kernels (FP32, and FP16 and BF16 storage rounded to nearest) are exactly equivariant under
the reflections of the D2Q9 lattice: a state that is mirror-symmetric about the x axis,
the y axis or the diagonal stays symmetric bit for bit (the fused kernel: about x and y).
The discrete step of Sec. 2 has these symmetries (M, the weights of Eq. (fint), m_eq, F_m
and both Q_m commute with the reflections); the test checks that no rounding breaks them,
since a rounding asymmetry of 1e-8 seeds the unstable modes of symmetric set-ups (the
translation of a liquid slab between walls)."""
import numpy as np
import pytest

from paper_2604_13407_gb300 import inputs as I
from paper_2604_13407_gb300 import lbm
from tests import gpu_cases as GC
from tests.setups import cs_case, cs_params

pytestmark = pytest.mark.gpu

# population index permutations of the reflections x -> -x, y -> -y, x <-> y
MIRROR_X = [0, 3, 2, 1, 4, 6, 5, 8, 7]
MIRROR_Y = [0, 1, 4, 3, 2, 8, 7, 6, 5]
MIRROR_D = [0, 2, 1, 4, 3, 5, 8, 7, 6]


def reflect(A, which):
    """Image of a population state [9][ny][nx] under a reflection of the lattice (nodes
    x -> nx - 1 - x, y -> ny - 1 - y, or transposed)."""
    if which == "x":
        return A[MIRROR_X][:, :, ::-1]
    if which == "y":
        return A[MIRROR_Y][:, ::-1, :]
    return np.transpose(A[MIRROR_D], (0, 2, 1))


# 16-bit storage rounded to nearest (stochastic rounding draws different random bits at
# mirror-image nodes, so it keeps a symmetric state symmetric only on average)
PRECS = [(lbm.F32, {}), (lbm.F16DEV, {"per_node_ref": 1, "storage_rounding": 0}),
         (lbm.BF16DEV, {"per_node_ref": 1, "storage_rounding": 0}), (lbm.F16DEV, {"storage_rounding": 0})]


@pytest.mark.parametrize("prec,kw", PRECS)
@pytest.mark.parametrize("scheme", [0, 1])
def test_channel_stays_mirror_symmetric(prec, kw, scheme):
    """The grid-aligned two-phase channel (4 x 128, walls in y, force along x): symmetric
    about the channel centre line after 3000 steps, two-pass kernel."""
    T, rg, rl = cs_case()
    p = cs_params(nx=4, ny=128, periodic_x=True, periodic_y=False, Fx=1e-7, scheme=scheme)
    c = GC.Case("c1", p, I.tanh_slab(4, 128, rl, rg, 64), 3000)
    s = GC.run_gpu(c, prec, **kw)
    A = s.get_state()
    assert np.all(np.isfinite(A))
    assert np.array_equal(A, reflect(A, "y"))


@pytest.mark.parametrize("prec,kw", PRECS)
@pytest.mark.parametrize("kernel", [lbm.KERNEL_TWO_PASS, lbm.KERNEL_FUSED])
def test_centred_droplet_keeps_all_mirror_symmetries(prec, kw, kernel):
    """A droplet at the centre of a periodic 256 x 256 box (no force), 200 steps.  The
    two-pass kernel keeps the symmetry about x, y and the diagonal; the fused kernel (the
    one the benchmark times) keeps x and y.  It evaluates the same expressions on packed
    pairs, and the compiler fuses some of the packed multiply-add chains of an x and a y
    quantity in only one of the two mirror-image expressions, so the diagonal symmetry
    holds there only to rounding."""
    T, rg, rl = cs_case()
    n = 256
    p = cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True, scheme=1)
    rho0 = I.droplet(n, n, rl, rg, 30, (n - 1) / 2, (n - 1) / 2, periodic_x=True)
    assert np.array_equal(rho0, rho0.T) and np.array_equal(rho0, rho0[::-1])
    s = GC.run_gpu(GC.Case("d", p, rho0, 200), prec, kernel, **kw)
    assert s.kernel_in_use == kernel
    A = s.get_state()
    assert np.all(np.isfinite(A))
    for w in ("x", "y", "d") if kernel == lbm.KERNEL_TWO_PASS else ("x", "y"):
        assert np.array_equal(A, reflect(A, w)), w
    if kernel == lbm.KERNEL_FUSED:
        assert np.abs(A - reflect(A, "d")).max() < 1e-3 * np.abs(A).max()


def test_falling_droplet_centred_stays_on_the_centre_line():
    """Buoyant droplet centred between walls at x = -1/2 and nx - 1/2 (x mirror symmetry,
    gravity along -y): the state stays symmetric about the centre line, so a migration
    off the centre line needs an asymmetric perturbation (here none)."""
    T, rg, rl = cs_case()
    p = cs_params(nx=48, ny=96, periodic_x=False, periodic_y=True, force_mode=1, Fy=-2e-5, scheme=1)
    rho0 = I.droplet(48, 96, rl, rg, 9, 23.5, 60.0, periodic_x=False)
    s = GC.run_gpu(GC.Case("fall", p, rho0, 1500), lbm.F32)
    A = s.get_state()
    assert np.array_equal(A, reflect(A, "x"))
