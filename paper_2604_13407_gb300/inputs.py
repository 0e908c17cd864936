"""Seeded synthetic inputs: initial density fields and wall geometries.

This module builds the inputs that both the CUDA library and the FP64 oracle are fed
in tests and benchmarks.  It holds none of the lattice Boltzmann arithmetic: only
initial profiles (Sec. 3 setups: tanh slabs, droplets, spinodal noise) and geometry
(solid masks, wall velocities, link wall fractions for interpolated bounce-back).

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), a counter-based
generator: value k of stream `seed` is splitmix64(seed * 2^32 + k), so any sample is
reproducible on any machine without numpy's generators.

Arrays are float64 / uint8 in row-major [ny][nx] order (x fastest).  Wall velocities
are [2][ny][nx]; link fractions q are [8][ny][nx] where q[d-1] at a fluid node is the
fraction of the link along e_d (D2Q9 numbering) at which the wall sits.
"""
import math

import numpy as np

# D2Q9 velocity set used only to trace links for the geometry (e_1..e_8)
_EX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
_EY = (0, 0, 1, 0, -1, 1, 1, -1, -1)

_MASK64 = (1 << 64) - 1


def splitmix64(counter):
    """SplitMix64 output for an array of uint64 counters."""
    z = (np.asarray(counter, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, n, lo=0.0, hi=1.0):
    """n uniform doubles in [lo, hi) from stream `seed` (53-bit mantissa)."""
    k = np.arange(n, dtype=np.uint64) + np.uint64((int(seed) << 32) & _MASK64)
    bits = splitmix64(k) >> np.uint64(11)
    return lo + (hi - lo) * (bits.astype(np.float64) * (1.0 / 9007199254740992.0))


def tanh_slab(nx, ny, rho_l, rho_g, width, axis="y", w=4.0, center=None):
    """Liquid slab of the given width between gas, tanh edges of width w (Sec. 3.1 setups).
    axis='y': the profile varies along y (flat interfaces parallel to x)."""
    n_len = ny if axis == "y" else nx
    c = (n_len - 1) / 2.0 if center is None else center
    d = np.arange(n_len, dtype=np.float64) - c
    L = float(width)
    prof = rho_g + 0.5 * (rho_l - rho_g) * (np.tanh(2.0 * (d + L / 2.0) / w) - np.tanh(2.0 * (d - L / 2.0) / w))
    if axis == "y":
        return np.repeat(prof[:, None], nx, axis=1)
    return np.repeat(prof[None, :], ny, axis=0)


def oblique_slab(n, rho_l, rho_g, width_alpha, w=4.0, period=None):
    """Slab whose profile depends on alpha = (x - y) (the 45-degree case of Sec. 2.1.2):
    index i = (x - y) mod period, liquid centred at period/2, width in alpha indices."""
    period = n if period is None else period
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None]
    i = np.mod(x - y, period).astype(np.float64)
    d = i - (period - 1) / 2.0
    L = float(width_alpha)
    return rho_g + 0.5 * (rho_l - rho_g) * (np.tanh(2.0 * (d + L / 2.0) / w) - np.tanh(2.0 * (d - L / 2.0) / w))


def oblique_band_walls(n, period=None, thickness=2):
    """Solid bands where (x - y) mod period < thickness: the 45-degree channel walls.
    Two solid diagonals are needed so that no population crosses a one-node wall."""
    period = n if period is None else period
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None]
    return (np.mod(x - y, period) < thickness).astype(np.uint8)


def droplet(nx, ny, rho_l, rho_g, radius, cx, cy, w=4.0, periodic_x=False, periodic_y=True):
    """Round droplet with a tanh edge (Sec. 3.3 setup)."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    dx = x - cx
    dy = y - cy
    if periodic_x:
        dx = (dx + nx / 2.0) % nx - nx / 2.0
    if periodic_y:
        dy = (dy + ny / 2.0) % ny - ny / 2.0
    r = np.sqrt(dx * dx + dy * dy)
    return 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (r - radius) / w)


def jittered_centre(seed, cx, cy, amp=4.0):
    """Droplet centre shifted by U(-amp, amp) in x and y from stream `seed`."""
    u = uniform(seed, 2, -amp, amp)
    return cx + float(u[0]), cy + float(u[1])


def spinodal(nx, ny, rho_mean, rel_amp=0.01, seed=5):
    """rho = rho_mean (1 + U(-rel_amp, rel_amp)) per node (the periodic spinodal workload)."""
    return rho_mean * (1.0 + uniform(seed, nx * ny, -rel_amp, rel_amp).reshape(ny, nx))


def _ray_circle(px, py, dx, dy, cx, cy, r):
    """Smallest t in (0, 1] with |p + t d - c| = r, or None."""
    fx, fy = px - cx, py - cy
    a = dx * dx + dy * dy
    b = 2.0 * (fx * dx + fy * dy)
    c = fx * fx + fy * fy - r * r
    disc = b * b - 4.0 * a * c
    if disc < 0.0:
        return None
    sq = math.sqrt(disc)
    best = None
    for t in ((-b - sq) / (2.0 * a), (-b + sq) / (2.0 * a)):
        if 1e-12 < t <= 1.0 + 1e-12 and (best is None or t < best):
            best = t
    return best


def annulus(nx, ny, r_in, r_out, u_wall_out=0.0, u_wall_in=0.0, cx=None, cy=None):
    """Concentric-cylinder geometry (Sec. 3.2 / annular shear): solid where r <= r_in or
    r >= r_out.  Returns (solid, wall_u, q): the solid nodes carry the tangential velocity
    of their cylinder (counter-clockwise for positive speeds) and q gives, for each
    fluid node and link crossing a circle, the fraction of the link at which it crosses."""
    cx = (nx - 1) / 2.0 if cx is None else cx
    cy = (ny - 1) / 2.0 if cy is None else cy
    x = np.arange(nx, dtype=np.float64)[None, :] - cx
    y = np.arange(ny, dtype=np.float64)[:, None] - cy
    r = np.sqrt(x * x + y * y)
    inner = r <= r_in
    outer = r >= r_out
    solid = (inner | outer).astype(np.uint8)
    with np.errstate(invalid="ignore", divide="ignore"):
        tx = np.where(r > 0, -y / r, 0.0)
        ty = np.where(r > 0, x / r, 0.0)
    speed = np.where(inner, u_wall_in, np.where(outer, u_wall_out, 0.0))
    wall_u = np.stack([speed * tx, speed * ty])
    q = np.full((8, ny, nx), 0.5)
    fluid_y, fluid_x = np.nonzero(solid == 0)
    for yy, xx in zip(fluid_y, fluid_x):
        for d in range(1, 9):
            xs, ys = xx + _EX[d], yy + _EY[d]
            if not (0 <= xs < nx and 0 <= ys < ny) or not solid[ys, xs]:
                continue
            px, py = xx - cx, yy - cy
            rad = r_in if inner[ys, xs] else r_out
            t = _ray_circle(px, py, _EX[d], _EY[d], 0.0, 0.0, rad)
            q[d - 1, yy, xx] = 0.5 if t is None else min(max(t, 1e-3), 1.0)
    return solid, wall_u, q
