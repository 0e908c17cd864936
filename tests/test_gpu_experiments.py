"""The paper's falling droplet (Sec. 3.3) on the GPU, its early stage: the improved scheme
accelerates the droplet faster than the original one (Sec. 3.3 reports this for
t* <= 50), and both fall on the centre line before any migration.  |g| = 2e-7, FP32,
t* up to 20 (tests/droplet_fall.py's set-up; about 1e6 steps per scheme on 256 x 2048)."""
import pytest

pytestmark = pytest.mark.gpu


def test_improved_scheme_accelerates_the_droplet_faster():
    from paper_2604_13407_gb300 import lbm
    from tests import droplet_fall as DF
    out = {}
    for scheme in (0, 1):
        samples, _ = DF.run(lbm, scheme, 2e-7, lbm.F32, 20.0, sample_every=5.0, kernel=lbm.KERNEL_TWO_PASS)
        out[scheme] = samples
    for scheme in (0, 1):
        for s in out[scheme]:
            assert s["U_c_star"] < 0.0  # falling
            assert abs(s["x_c_over_W"] - 0.5) < 0.01  # still on the centre line
    u0 = [abs(s["U_c_star"]) for s in out[0]]
    u1 = [abs(s["U_c_star"]) for s in out[1]]
    assert all(b > a for a, b in zip(u0, u1)), (u0, u1)
    assert u1[-1] > 1.02 * u0[-1], (u0, u1)
    # still accelerating at t* = 20
    assert u0[-1] > u0[-2] and u1[-1] > u1[-2]
