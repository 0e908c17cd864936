"""Analytic and semi-analytic references that pin the FP64 oracle (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Each function restates a relation the paper (Huang, Huang
& Li 2026) or textbook thermodynamics fixes; none of them calls the C oracle.

  p_eos, psi, dpsi          EOS of Sec. 3 (van der Waals) and Carnahan-Starling (Sec. 2)
  maxwell                   Maxwell equal-area construction (mentioned in Sec. 3.1)
  mechanical_stability      coexistence densities of the mechanical stability
                            condition, Eq. (1) of Sec. 1, weight psi'/psi^(1+eps)
  poiseuille_theory         integral of Eq. (u.plane) with a given density profile
  err_norm                  Err of Sec. 3.1
  fde_aligned_residual      residual of Eq. (fde.ali)
  fde_oblique_residual      residual of Eq. (fde.obl)
  ali3_residual             residual of Eq. (ali.3)
  fint_closed_form          Eq. (obl.10)
"""
import math

import numpy as np
from scipy import integrate, linalg, optimize


# ----------------------------------------------------------------- EOS -----

def p_eos(rho, eos, a, b, R, T, K=1.0):
    """van der Waals (Sec. 3) or Carnahan-Starling pressure."""
    rho = np.asarray(rho, dtype=np.float64)
    if eos == 0:
        return K * (rho * R * T / (1.0 - b * rho) - a * rho * rho)
    eta = b * rho / 4.0
    return K * (rho * R * T * (1.0 + eta + eta**2 - eta**3) / (1.0 - eta) ** 3 - a * rho * rho)


def dp_eos(rho, eos, a, b, R, T, K=1.0):
    """d p / d rho, differentiated by hand from p_eos."""
    rho = np.asarray(rho, dtype=np.float64)
    if eos == 0:
        return K * (R * T / (1.0 - b * rho) + rho * R * T * b / (1.0 - b * rho) ** 2 - 2.0 * a * rho)
    eta = b * rho / 4.0
    g = (1.0 + eta + eta**2 - eta**3) / (1.0 - eta) ** 3
    # d g / d eta = [(1 + 2 eta - 3 eta^2)(1 - eta) + 3 (1 + eta + eta^2 - eta^3)] / (1 - eta)^4
    dg = ((1.0 + 2.0 * eta - 3.0 * eta**2) * (1.0 - eta)
          + 3.0 * (1.0 + eta + eta**2 - eta**3)) / (1.0 - eta) ** 4
    return K * (R * T * g + rho * R * T * dg * b / 4.0 - 2.0 * a * rho)


def psi(rho, eos, a, b, R, T, K=1.0, G=-1.0):
    """Sec. 2: psi = sqrt(2 (p_EOS - rho/3) / G)."""
    return np.sqrt(2.0 * (p_eos(rho, eos, a, b, R, T, K) - np.asarray(rho) / 3.0) / G)


def dpsi(rho, eos, a, b, R, T, K=1.0, G=-1.0):
    """d psi / d rho = (p' - 1/3) / (G psi)."""
    return (dp_eos(rho, eos, a, b, R, T, K) - 1.0 / 3.0) / (G * psi(rho, eos, a, b, R, T, K, G))


def cs_critical(a, b, R):
    """Carnahan-Starling critical point with the usual four-digit constants: T_c =
    0.3773 a/(b R) and the critical packing fraction eta_c = b rho_c/4 = 0.1304, i.e.
    rho_c = 0.5218/b (0.1304 for the b = 4 of the pseudopotential literature).
    tests/test_eos_pins.py finds both from the oracle's compiled p_EOS."""
    return 0.3773 * a / (b * R), 4.0 * 0.1304 / b


def vdw_critical(a, b, R):
    """Sec. 3: T_cr = 8a/(27 R b), rho_cr = 1/(3b)."""
    return 8.0 * a / (27.0 * R * b), 1.0 / (3.0 * b)


# ---------------------------------------------------------- coexistence ----

def _spinodal(eos, a, b, R, T, K, rho_hi):
    """Local max and min of p(rho) on (0, rho_hi): the two spinodal densities."""
    xs = np.linspace(1e-6, rho_hi, 20001)
    dp = dp_eos(xs, eos, a, b, R, T, K)
    sign_change = np.nonzero(np.diff(np.sign(dp)))[0]
    if len(sign_change) < 2:
        raise ValueError("no van der Waals loop at this temperature")
    r1 = optimize.brentq(lambda r: dp_eos(r, eos, a, b, R, T, K), xs[sign_change[0]], xs[sign_change[0] + 1])
    r2 = optimize.brentq(lambda r: dp_eos(r, eos, a, b, R, T, K), xs[sign_change[1]], xs[sign_change[1] + 1])
    return r1, r2


def _coexistence(weight, eos, a, b, R, T, K, rho_hi):
    """Solve p(rho_g) = p(rho_l) = p_sat and int_{rho_g}^{rho_l} (p_sat - p) weight drho = 0
    by a one-dimensional root search on p_sat between the spinodal pressures."""
    s1, s2 = _spinodal(eos, a, b, R, T, K, rho_hi)
    p_lo = float(p_eos(s2, eos, a, b, R, T, K))
    p_hi = float(p_eos(s1, eos, a, b, R, T, K))

    def roots(ps):
        rg = optimize.brentq(lambda r: p_eos(r, eos, a, b, R, T, K) - ps, 0.0, s1)
        rl = optimize.brentq(lambda r: p_eos(r, eos, a, b, R, T, K) - ps, s2, rho_hi)
        return rg, rl

    def area(ps):
        rg, rl = roots(ps)
        val, _ = integrate.quad(lambda r: (ps - p_eos(r, eos, a, b, R, T, K)) * weight(r),
                                rg, rl, limit=400, epsabs=1e-15, epsrel=1e-13)
        return val

    lo = max(p_lo, 0.0) + 1e-9 * abs(p_hi)
    hi = p_hi - 1e-9 * abs(p_hi)
    grid = np.linspace(lo, hi, 65)
    vals = [area(g) for g in grid]
    k = next((j for j in range(64) if np.sign(vals[j]) != np.sign(vals[j + 1])), None)
    if k is None:
        raise ValueError("no coexistence with a positive saturation pressure")
    ps = optimize.brentq(area, grid[k], grid[k + 1], xtol=1e-18, rtol=1e-14, maxiter=500)
    rg, rl = roots(ps)
    return rg, rl, ps


def maxwell(eos, a, b, R, T, K=1.0, rho_hi=None):
    """Thermodynamic coexistence: equal area in the specific-volume plane, weight 1/rho^2."""
    if rho_hi is None:
        rho_hi = (0.999 / b) if eos == 0 else (3.9 / b)
    return _coexistence(lambda r: 1.0 / (r * r), eos, a, b, R, T, K, rho_hi)


def mechanical_stability(epsilon, eos, a, b, R, T, K=1.0, rho_hi=None, G=-1.0):
    """Eq. (1): int (p_sat - p_EOS) psi'/psi^(1+eps) drho = 0 (independent of G).
    The liquid branch is searched only where psi is real (p_EOS < rho/3)."""
    if rho_hi is None:
        rho_hi = (0.999 / b) if eos == 0 else (3.9 / b)
        xs = np.linspace(1e-6, rho_hi, 40001)
        bad = np.nonzero(p_eos(xs, eos, a, b, R, T, K) - xs / 3.0 >= 0.0)[0]
        if len(bad):
            rho_hi = xs[bad[0] - 1]
    w = lambda r: dpsi(r, eos, a, b, R, T, K, G) / psi(r, eos, a, b, R, T, K, G) ** (1.0 + epsilon)
    return _coexistence(w, eos, a, b, R, T, K, rho_hi)


# ---------------------------------------------------------- flow profiles --

def nu_of_rho(rho, tau_l, tau_g, rho_l, rho_g):
    """Kinematic viscosity nu = (tau - 1/2)/3, interpolated linearly in rho (clamped)."""
    nu_l, nu_g = (tau_l - 0.5) / 3.0, (tau_g - 0.5) / 3.0
    if tau_l == tau_g:
        return np.full_like(np.asarray(rho, dtype=np.float64), nu_l)
    w = np.clip((np.asarray(rho) - rho_g) / (rho_l - rho_g), 0.0, 1.0)
    return nu_g + w * (nu_l - nu_g)


def poiseuille_theory(rho_nodes, F, nu_fn, spacing=1.0, sub=400):
    """Integrate Eq. (u.plane), d/dn (rho nu du/dn) = -F, across a channel whose nodes sit
    at n_j = (j + 1/2) spacing for j = 0..N-1 with walls (u = 0) at n = 0 and n = N spacing.
    The density is interpolated linearly between nodes (held constant in the half cells
    next to the walls).  The shear stress of a symmetric channel vanishes at the centre
    line, so rho nu du/dn = -F (n - n_c) and u(n) = int_0^n -F (s - n_c)/(rho nu)(s) ds."""
    rho_nodes = np.asarray(rho_nodes, dtype=np.float64)
    N = len(rho_nodes)
    width = N * spacing
    nodes = (np.arange(N) + 0.5) * spacing
    s = np.linspace(0.0, width, N * sub + 1)
    rho_s = np.interp(s, nodes, rho_nodes)
    mu = rho_s * nu_fn(rho_s)
    # centre line: zero of the integral of the stress across the channel is at the
    # symmetric midpoint only when mu is symmetric; solve for the stress offset so that
    # u vanishes on both walls: u(width) = int -F (s - c)/mu ds = 0
    i1 = integrate.trapezoid(s / mu, s)
    i0 = integrate.trapezoid(1.0 / mu, s)
    c = i1 / i0
    g = -F * (s - c) / mu
    u = integrate.cumulative_trapezoid(g, s, initial=0.0)
    return np.interp(nodes, s, u)


def annular_theory(r_nodes, rho_nodes, F_fn, nu_fn, R_i, R_o, sub=400):
    """Integrate Eq. (u.annular), (1/r^2) d/dr [rho nu r^3 d(u/r)/dr] = -F(r), between
    no-slip cylinders at r = R_i and R_o, with the density interpolated linearly between
    the sampled radii r_nodes (held constant between the outermost samples and the walls).
    With mu = rho nu and G(r) = int_{R_i}^r s^2 F(s) ds the first integral is
    mu r^3 d(u/r)/dr = C - G(r), so u/r = int_{R_i}^r (C - G)/(mu s^3) ds, and C makes u vanish
    at R_o.  Returns u at r_nodes."""
    r_nodes = np.asarray(r_nodes, dtype=np.float64)
    rho_nodes = np.asarray(rho_nodes, dtype=np.float64)
    s = np.linspace(R_i, R_o, (len(r_nodes) + 1) * sub + 1)
    rho_s = np.interp(s, r_nodes, rho_nodes)
    mu = rho_s * nu_fn(rho_s)
    G = integrate.cumulative_trapezoid(s * s * F_fn(s), s, initial=0.0)
    i1 = integrate.trapezoid(1.0 / (mu * s**3), s)
    iG = integrate.trapezoid(G / (mu * s**3), s)
    C = iG / i1
    w = integrate.cumulative_trapezoid((C - G) / (mu * s**3), s, initial=0.0)
    return np.interp(r_nodes, s, s * w)


def err_norm(u_sim, u_th):
    """Err of Sec. 3.1: sqrt(sum (u_sim - u_th)^2 / sum u_th^2)."""
    u_sim = np.asarray(u_sim)
    u_th = np.asarray(u_th)
    return float(np.sqrt(np.sum((u_sim - u_th) ** 2) / np.sum(u_th**2)))


# --------------------------------------------------- discrete identities ---

def ali3_residual(f_par_plus, f_par_minus, rho, u_par, F_par, Q_par, s_q):
    """Eq. (ali.3): f_(+) - f_(-) = 2/3 rho u + (2 - s_q)/(3 s_q) F - Q/3 along the flow
    direction at steady state (f_(+), f_(-) the axis populations along and against the flow,
    F the total force along the flow, Q the source term of the flow-direction q moment)."""
    return (f_par_plus - f_par_minus) - (2.0 / 3.0 * rho * u_par
                                         + (2.0 - s_q) / (3.0 * s_q) * F_par - Q_par / 3.0)


def fde_aligned_residual(rho, Fn, u, Q, F_dri, nu):
    """Eq. (fde.ali) at interior indices 1..N-2 (profile index i normal to the flow,
    Fn the pairwise force along +i, u and Q along the flow).  Returns LHS - RHS."""
    rho, Fn, u, Q = map(np.asarray, (rho, Fn, u, Q))
    lhs = ((rho[:-2] + 1.5 * Fn[:-2]) * u[:-2] + (rho[2:] - 1.5 * Fn[2:]) * u[2:]
           - 2.0 * rho[1:-1] * u[1:-1] + (Q[:-2] + Q[2:] - 2.0 * Q[1:-1]))
    return lhs + F_dri / nu


def lb_ana_aligned(rho, Fn, X, kq, F_dri, nu, u_ends=None):
    """"LB-ana" of Sec. 3.1: the velocity profile that solves Eq. (fde.ali) for a given
    steady density profile, with Q_m,6 = kq X u (Eq. (qm6.ali): kq = 3 epsilon / 8 for the
    improved scheme; the original scheme has Q_m,6 = 0, kq = 0).  Fn is the pairwise
    force along the profile, X = dt^2 F_hat^2 / psi_hat^2 = Fn^2 / (-G psi^2).  Row i reads
      (rho + 3/2 Fn + kq X)^{i-1} u^{i-1} + (rho - 3/2 Fn + kq X)^{i+1} u^{i+1}
        - 2 (rho + kq X)^i u^i = -F_dri / nu.
    The walls are not part of the equation: with u_ends = None each end row sees a mirror
    ghost node (u = -u of the end node, its coefficients those of the end node with Fn
    reversed), a half-way no-slip wall; with u_ends = (u_0, u_{N-1}) the end values are
    given and the interior rows are solved."""
    rho, Fn, X = (np.asarray(v, dtype=np.float64) for v in (rho, Fn, X))
    N = len(rho)
    sub = rho[:-1] + 1.5 * Fn[:-1] + kq * X[:-1]  # row i, column i - 1
    sup = rho[1:] - 1.5 * Fn[1:] + kq * X[1:]     # row i, column i + 1
    diag = -2.0 * (rho + kq * X)
    diag[0] -= rho[0] - 1.5 * Fn[0] + kq * X[0]
    diag[-1] -= rho[-1] + 1.5 * Fn[-1] + kq * X[-1]
    b = np.full(N, -F_dri / nu)
    if u_ends is not None:
        u0, u1 = u_ends
        bi = b[1:-1].copy()
        bi[0] -= sub[0] * u0
        bi[-1] -= sup[-1] * u1
        u = np.empty(N)
        u[0], u[-1] = u0, u1
        u[1:-1] = _tridiagonal(sub[1:-1], diag[1:-1], sup[1:-1], bi)
        return u
    return _tridiagonal(sub, diag, sup, b)


def _tridiagonal(sub, diag, sup, b):
    """Solve the tridiagonal system with sub-, main and super-diagonals (a library banded
    solver, LU with partial pivoting)."""
    ab = np.zeros((3, len(diag)))
    ab[0, 1:] = sup
    ab[1] = diag
    ab[2, :-1] = sub
    return linalg.solve_banded((1, 1), ab, b)


def lb_ana_oblique(rho, Fx, X, K, F_dri, nu):
    """Eq. (fde.obl) solved for u_beta along alpha (node spacing dx/sqrt 2), with
    Q_m,4+6 = -2 sqrt 2 K X u_beta (Eq. (obl.11) written with u_x + u_y = sqrt 2 u_beta;
    the improved scheme has K = (24 epsilon - 15)/32, the original K = 0).  Fx is the x
    component of the pairwise force (Eq. (obl.10)), X = dt^2 F_hat_x^2 / psi_hat^2.  Since
    -sqrt 2/4 times the second difference of Q_m,4+6 is + K times that of X u_beta, row i reads
      (rho + 3/2 Fx + K X)^{i-1} u^{i-1} + (rho - 3/2 Fx + K X)^{i+1} u^{i+1}
        - 2 (rho + K X)^i u^i = -F_dri / (2 nu).
    Each end row sees a mirror ghost node (u = -u of the end node, Fx reversed): a
    half-way no-slip wall."""
    rho, Fx, X = (np.asarray(v, dtype=np.float64) for v in (rho, Fx, X))
    sub = rho[:-1] + 1.5 * Fx[:-1] + K * X[:-1]
    sup = rho[1:] - 1.5 * Fx[1:] + K * X[1:]
    diag = -2.0 * (rho + K * X)
    diag[0] -= rho[0] - 1.5 * Fx[0] + K * X[0]
    diag[-1] -= rho[-1] + 1.5 * Fx[-1] + K * X[-1]
    return _tridiagonal(sub, diag, sup, np.full(len(rho), -F_dri / (2.0 * nu)))


def fde_oblique_residual(rho, Fx, u_beta, Q46, F_dri, nu):
    """Eq. (fde.obl) at interior indices 1..N-2, with i the index along alpha
    (node spacing dx/sqrt 2), Fx the x component of the pairwise force, u_beta the
    velocity along beta and Q46 = Q_4 + Q_6.  Returns LHS - RHS."""
    rho, Fx, u_beta, Q46 = map(np.asarray, (rho, Fx, u_beta, Q46))
    lhs = ((rho[:-2] + 1.5 * Fx[:-2]) * u_beta[:-2] + (rho[2:] - 1.5 * Fx[2:]) * u_beta[2:]
           - 2.0 * rho[1:-1] * u_beta[1:-1]
           - math.sqrt(2.0) / 4.0 * (Q46[:-2] + Q46[2:] - 2.0 * Q46[1:-1]))
    return lhs + F_dri / (2.0 * nu)


def fint_closed_form(psi_hat, oblique=False):
    """Eq. (obl.10) with dt = 1 on a periodic 1-D profile of the rescaled pseudopotential
    psi_hat = sqrt(-G) psi: the pairwise force component along the profile (aligned) or
    its x component (oblique, profile index along alpha)."""
    p = np.asarray(psi_hat)
    if not oblique:
        return p * (np.roll(p, -1) - np.roll(p, 1)) / 2.0
    return p * (np.roll(p, -2) + 4.0 * np.roll(p, -1) - 4.0 * np.roll(p, 1) - np.roll(p, 2)) / 12.0
