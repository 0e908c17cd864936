"""Pins of the "Theory" integrators of Secs. 3.1-3.2 (oracle/analytic.py) against closed
forms: Eq. (u.plane) for a uniform and for a three-layer channel, Eq. (u.annular) for a
uniform annulus with the driving force F_o r^2 / R_o^2."""
import numpy as np

from oracle import analytic as A


def test_plane_theory_uniform_is_the_parabola():
    """d/dn (mu du/dn) = -F with u = 0 at n = 0, W: u = F n (W - n) / (2 mu)."""
    N, F, nu, rho = 101, 3e-7, 0.1, 2.5
    u = A.poiseuille_theory(np.full(N, rho), F, lambda r: np.full_like(r, nu))
    n = np.arange(N) + 0.5
    exact = F * n * (N - n) / (2.0 * rho * nu)
    assert np.abs(u - exact).max() <= 1e-9 * exact.max()


def test_plane_theory_three_layers():
    """Gas layers of mu_g on either side of a liquid layer of mu_l (symmetric): the stress is
    -F (n - c), so u(n) = int_0^n F (c - s) / mu(s) ds piecewise.  The sampled density
    jumps over one node spacing, an O(1/N) error, so the pin uses many nodes."""
    N, F, nu = 4000, 1e-7, 0.2
    n = np.arange(N) + 0.5
    c, h = N / 2.0, N / 4.0
    rho_l, rho_g = 7.0, 0.125
    rho = np.where(np.abs(n - c) < h, rho_l, rho_g)
    u = A.poiseuille_theory(rho, F, lambda r: np.full_like(r, nu))
    mg, ml = rho_g * nu, rho_l * nu
    prim = lambda s: F * (c * s - 0.5 * s * s)  # int F (c - s) ds
    a = c - h
    nn = np.minimum(n, N - n)  # symmetric
    exact = np.where(nn < a, prim(nn) / mg, prim(a) / mg + (prim(nn) - prim(a)) / ml)
    assert np.abs(u - exact).max() <= 1e-3 * exact.max()
    # the plug: the liquid moves almost uniformly at the speed the gas layers allow
    assert abs(u[N // 2] - exact[N // 2]) <= 1e-3 * exact[N // 2]


def test_annular_theory_uniform_closed_form():
    """mu r^3 (u/r)' = C - F_o (r^5 - R_i^5) / (5 R_o^2) integrates to
    u/r = -F_o r^3 / (15 mu R_o^2) - C' / r^2 + D, with C', D fixed by u(R_i) = u(R_o) = 0."""
    R_i, R_o, F_o, rho, nu = 64.0, 256.0, 3e-5, 1.3, 0.1
    mu = rho * nu
    r = np.linspace(R_i + 0.5, R_o - 0.5, 192)
    u = A.annular_theory(r, np.full_like(r, rho), lambda s: F_o * s * s / R_o**2,
                         lambda x: np.full_like(x, nu), R_i, R_o)
    g = lambda x: -F_o * x**3 / (15.0 * mu * R_o**2)
    M = np.array([[-1.0 / R_i**2, 1.0], [-1.0 / R_o**2, 1.0]])
    cp, d = np.linalg.solve(M, [-g(R_i), -g(R_o)])
    exact = r * (g(r) - cp / r**2 + d)
    assert np.abs(u - exact).max() <= 1e-8 * np.abs(exact).max()
    assert exact.max() > 0  # counter-clockwise force, counter-clockwise flow


def test_annular_theory_scales_with_viscosity_and_force():
    """Linear in F and in 1/(rho nu): a wrong power anywhere breaks one of the two."""
    R_i, R_o = 10.0, 40.0
    r = np.linspace(R_i + 0.5, R_o - 0.5, 30)
    rho = 1.0 + 0.5 * np.tanh((r - 20.0) / 2.0)
    base = A.annular_theory(r, rho, lambda s: 1e-5 * s * s / R_o**2, lambda x: np.full_like(x, 0.1), R_i, R_o)
    twice = A.annular_theory(r, rho, lambda s: 2e-5 * s * s / R_o**2, lambda x: np.full_like(x, 0.1), R_i, R_o)
    visc = A.annular_theory(r, rho, lambda s: 1e-5 * s * s / R_o**2, lambda x: np.full_like(x, 0.2), R_i, R_o)
    assert np.allclose(twice, 2.0 * base, rtol=1e-12)
    assert np.allclose(visc, 0.5 * base, rtol=1e-12)
