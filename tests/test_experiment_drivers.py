"""Host logic of the experiment drivers, on synthetic inputs (no GPU): the falling-droplet
summary (terminal velocity over the last 15 % of the run, migration onset) and the
annulus geometry (the two rays along which Sec. 3.2 compares profiles, and the angular
driving force F_o r^2 / R_o^2)."""
import math

import numpy as np

from tests import annular as AN
from tests import droplet_fall as DF


def samples(t_star, u_star, xc):
    return [{"t_star": t, "U_c_star": u, "x_c_over_W": x, "max_u": 0.1} for t, u, x in zip(t_star, u_star, xc)]


def test_droplet_summary_terminal_velocity_and_no_migration():
    t = np.arange(1, 201, dtype=float)
    u = -1.0 + 0.5 * np.exp(-t / 20.0)  # falling, approaching -1
    s = DF.summarise(samples(t, u, np.full_like(t, 0.5)), 1, 0.5e-7)
    assert abs(s["terminal_U_c_star"] - np.abs(u[t >= 0.85 * 200]).mean()) < 1e-15
    assert s["migration_t_star"] is None and s["U_c_star_at_migration"] is None
    assert s["paper_terminal_U_c_star"] == 1.0104


def test_droplet_summary_migration_onset():
    """The onset is the last sample within 1 % of the centre line before the centre of
    mass leaves 5 %."""
    t = np.arange(1, 101, dtype=float)
    xc = np.where(t < 40, 0.5, 0.5 - 0.004 * (t - 39) ** 2)  # leaves the centre after t* = 39
    u = -np.minimum(t / 30.0, 1.5)
    s = DF.summarise(samples(t, u, np.clip(xc, 0.27, 0.5)), 0, 2e-7)
    first_off = t[np.abs(np.clip(xc, 0.27, 0.5) - 0.5) > 0.05][0]
    assert s["migration_t_star"] < first_off
    near = t[(t < first_off) & (np.abs(np.clip(xc, 0.27, 0.5) - 0.5) < 0.01)]
    assert s["migration_t_star"] == near[-1]
    assert abs(s["U_c_star_at_migration"] - abs(u[int(near[-1]) - 1])) < 1e-15
    assert abs(s["final_x_c_over_W"] - 0.27) < 1e-12


def test_annulus_rays_and_force_field():
    solid, q, x, y, r = AN.geometry()
    rays = AN.rays(r)
    idx, rr, (tx, ty) = rays["horizontal"]
    assert np.all((rr > AN.R_I) & (rr < AN.R_O))
    assert np.all(solid[idx[:, 0], idx[:, 1]] == 0)
    assert np.allclose(rr, idx[:, 1] - AN.C) and (tx, ty) == (0.0, 1.0)
    idx, rr, (tx, ty) = rays["diagonal"]
    assert np.allclose(rr, (idx[:, 0] - AN.C) * math.sqrt(2.0))
    assert np.all(solid[idx[:, 0], idx[:, 1]] == 0)
    assert abs(tx * tx + ty * ty - 1.0) < 1e-15 and tx < 0 < ty
    F = AN.force_field(x, y, r, solid)
    mag = np.hypot(F[0], F[1])
    fluid = solid == 0
    assert np.allclose(mag[fluid], AN.F_O * r[fluid] ** 2 / AN.R_O**2)
    # tangential and counter-clockwise: F . r = 0 and (r x F)_z > 0
    assert np.abs(F[0] * x + F[1] * y)[fluid].max() < 1e-12 * AN.F_O * AN.R_O
    assert np.all((x * F[1] - y * F[0])[fluid & (r > 1)] > 0)
    assert np.all(mag[solid == 1] == 0.0)
