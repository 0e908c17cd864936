"""The library's "LB-ana" (lbm_lb_ana, Sec. 3.1): the velocity profile the step predicts for a
given density profile, from Eq. (fde.ali) (grid-aligned) or Eq. (fde.obl) (45 degrees).  Runs on
the host, so these are CPU tests.

Pins: single-phase flow, where Eq. (fde.ali) reduces to the second-order finite-difference
Poisson equation whose solution with half-way walls is a closed-form parabola (the same for
Eq. (fde.obl) with its dx/sqrt 2 node spacing).  Parity: against the oracle's own solvers
(oracle/analytic.py lb_ana_aligned, lb_ana_oblique, pinned by tests/test_table1_golden.py and
tests/test_oblique_k.py) on the oracle's converged Table 1 profiles and 45-degree profiles."""
import json
import math
import pathlib

import numpy as np
import pytest

from oracle import analytic as A
from paper_2604_13407_gb300 import lbm
from tests.setups import vdw_params

GOLD = pathlib.Path(__file__).parent / "golden"
ALIGNED = json.loads((GOLD / "table1_aligned_oracle.json").read_text())["rows"]
OBLIQUE = json.loads((GOLD / "oblique_profiles.json").read_text())["rows"]
F_DRIVE = 2e-7


def lib_params(op, tau, scheme):
    fields = ("eos", "a", "b", "R", "T", "K_eos", "G", "k1", "k2", "rho_l", "rho_g", "rho_s")
    p = lbm.default_params(**{f: getattr(op, f) for f in fields})
    p.tau_l = p.tau_g = tau
    p.scheme = scheme
    return p


@pytest.mark.parametrize("oblique", [False, True])
def test_single_phase_profile_is_the_exact_parabola(oblique):
    """Uniform density, rho_s = rho: no pairwise force, no source term, and the equation is
    the second-order finite-difference Poisson equation rho nu u'' = -F with node spacing h
    (1 aligned, 1/sqrt 2 at 45 degrees).  Its solution with the mirror (antisymmetric) ghost
    nodes of half-way walls at s = 0 and s = W = n h is the parabola through the walls
    shifted by the ghost's interpolation slip:
        u_i = F/(2 rho nu) (s_i (W - s_i) + h^2/4),  s_i = (i + 1/2) h,
    since a quadratic satisfies the three-point difference exactly and u_-1 + u_0 = 0 fixes
    the constant.  Round-off only."""
    op = vdw_params(1.0, 0.65)
    rho0 = 2.0
    op.rho_s = rho0
    n, tau = 41, 0.9
    p = lib_params(op, tau, lbm.IMPROVED)
    u = lbm.lb_ana(p, np.full(n, rho0), F_DRIVE, oblique=oblique)
    nu = (tau - 0.5) / 3.0
    h = 1.0 / math.sqrt(2.0) if oblique else 1.0
    s = (np.arange(n) + 0.5) * h
    exact = F_DRIVE / (2.0 * rho0 * nu) * (s * (n * h - s) + h * h / 4.0)
    assert np.abs(u - exact).max() <= 1e-12 * exact.max(), np.abs(u - exact).max() / exact.max()


def _aligned_inputs(row):
    rho = np.array(row["profiles"]["rho"])
    op = vdw_params(row["epsilon"], row["T_r"], nx=1, ny=len(rho))
    psi_hat = np.sqrt(-op.G) * A.psi(rho, 0, op.a, op.b, op.R, op.T, op.K_eos, op.G)
    psi_wall = np.sqrt(-op.G) * A.psi(op.rho_s, 0, op.a, op.b, op.R, op.T, op.K_eos, op.G)
    padded = np.concatenate([[psi_wall], psi_hat, [psi_wall]])
    Fn = psi_hat * (padded[2:] - padded[:-2]) / 2.0
    return op, rho, Fn, Fn**2 / psi_hat**2, np.array(row["profiles"]["u"])


@pytest.mark.parametrize("key", [(e, s) for e in (0.0, 1.0, 2.0) for s in ("original", "improved")],
                         ids=lambda k: "eps%g-%s" % k)
def test_aligned_matches_the_oracle_on_table1_profiles(key):
    """Eq. (fde.ali) on the oracle's converged tau = 1.5 Table 1 densities: the library (force
    from the density and psi(rho_s) at the walls) against the oracle's solver (force computed
    the same way by the test): 1e-9 of the profile's maximum; both reproduce the simulated
    velocity to 2e-4 of its maximum."""
    eps, scheme = key
    row = next(r for r in ALIGNED if r["epsilon"] == eps and r["tau"] == 1.5 and r["scheme"] == scheme)
    op, rho, Fn, X, u_sim = _aligned_inputs(row)
    kq = 3.0 * eps / 8.0 if scheme == "improved" else 0.0
    u_or = A.lb_ana_aligned(rho, Fn, X, kq, F_DRIVE, (1.5 - 0.5) / 3.0)
    p = lib_params(op, 1.5, lbm.IMPROVED if scheme == "improved" else lbm.ORIGINAL)
    u_lib = lbm.lb_ana(p, rho, F_DRIVE)
    assert np.abs(u_lib - u_or).max() <= 1e-9 * np.abs(u_or).max()
    assert np.abs(u_lib - u_sim).max() <= 2e-4 * np.abs(u_sim).max()
    # the force given explicitly gives the same profile
    assert np.abs(lbm.lb_ana(p, rho, F_DRIVE, f_int=Fn) - u_or).max() <= 1e-9 * np.abs(u_or).max()


def _oblique_inputs(row):
    rho_p = np.array(row["rho_alpha"])
    op = vdw_params(row["epsilon"], row["T_r"], nx=4, ny=4)
    psi_hat = np.sqrt(-op.G) * A.psi(rho_p, 0, op.a, op.b, op.R, op.T, op.K_eos, op.G)
    Fx = A.fint_closed_form(psi_hat, oblique=True)
    idx = (np.arange(len(rho_p)) + int(np.argmin(rho_p))) % len(rho_p)
    return op, rho_p[idx], Fx[idx], (Fx**2 / psi_hat**2)[idx]


@pytest.mark.parametrize("scheme", ["original", "improved"])
@pytest.mark.parametrize("row", OBLIQUE, ids=lambda r: "eps%g" % r["epsilon"])
def test_oblique_matches_the_oracle(row, scheme):
    """Eq. (fde.obl) on the oracle's steady 45-degree profiles, the force of Eq. (obl.10) given
    to both: the library against the oracle's solver with K = (24 eps - 15)/32 (improved) or
    0 (original), 1e-9 of the profile's maximum."""
    op, rho, Fx, X = _oblique_inputs(row)
    eps = row["epsilon"]
    K = (24.0 * eps - 15.0) / 32.0 if scheme == "improved" else 0.0
    u_or = A.lb_ana_oblique(rho, Fx, X, K, F_DRIVE, (1.5 - 0.5) / 3.0)
    p = lib_params(op, 1.5, lbm.IMPROVED if scheme == "improved" else lbm.ORIGINAL)
    u_lib = lbm.lb_ana(p, rho, F_DRIVE, oblique=True, f_int=Fx)
    assert np.abs(u_lib - u_or).max() <= 1e-9 * np.abs(u_or).max()


def test_improved_source_removes_the_aligned_oscillation():
    """Sec. 3.1's finding through the library alone: on the epsilon = 2 Table 1 density the
    original scheme's LB-ana profile is far from "Theory" (Eq. (u.plane)) and the improved
    one is close (Err 0.129 -> 1.3e-3 in the simulations)."""
    row = next(r for r in ALIGNED if r["epsilon"] == 2.0 and r["tau"] == 1.5 and r["scheme"] == "improved")
    op, rho, _, _, _ = _aligned_inputs(row)
    th = A.poiseuille_theory(rho, F_DRIVE, lambda r: np.full_like(r, (1.5 - 0.5) / 3.0))
    e = {s: A.err_norm(lbm.lb_ana(lib_params(op, 1.5, s), rho, F_DRIVE), th) for s in (lbm.ORIGINAL, lbm.IMPROVED)}
    assert e[lbm.IMPROVED] * 20 < e[lbm.ORIGINAL], e


def test_rejects_invalid_input():
    op = vdw_params(1.0, 0.65)
    p = lib_params(op, 0.8, lbm.IMPROVED)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lb_ana(p, np.full(2, 2.0), F_DRIVE)
    assert e.value.status == 1
    p.tau_g = 0.6
    with pytest.raises(lbm.LbmError) as e:
        lbm.lb_ana(p, np.full(10, 2.0), F_DRIVE)
    assert e.value.status == 1 and "tau" in str(e.value)
