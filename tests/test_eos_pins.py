"""Pins of the oracle's equations of state (Sec. 2, Sec. 3) by their critical points.

The critical point of an EOS is where the isotherm has a horizontal inflection,
dp/drho = d2p/drho2 = 0.  It is found here numerically from the oracle's own compiled
p_EOS (lbm_oracle.c, through ctypes), with finite differences and root finding only, and
compared with the published values:
  - van der Waals (Sec. 3): T_cr = 8a/(27 R b), rho_cr = 1/(3b), for any K_EOS;
  - Carnahan-Starling (standard form, eta = b rho/4): T_c = 0.3773 a/(b R) and the
    critical packing fraction eta_c = b rho_c/4 = 0.1304 (four digits; with the b = 4 of
    the pseudopotential literature, rho_c = 0.1304).
A wrong exponent of (1 - eta), a dropped term of the numerator, a wrong b/4 or a wrong
sign of the attraction term moves the critical point and fails these tests."""
import math

import pytest
from scipy.optimize import brentq

from oracle import oracle as O


def _params(eos, a, b, R, K=1.0, T=1.0):
    return O.Params(eos=eos, a=a, b=b, R=R, T=T, K_eos=K)


def _d1(p, rho, h):
    return (-p(rho + 2 * h) + 8 * p(rho + h) - 8 * p(rho - h) + p(rho - 2 * h)) / (12 * h)


def _d2(p, rho, h):
    return (-p(rho + 2 * h) + 16 * p(rho + h) - 30 * p(rho) + 16 * p(rho - h) - p(rho - 2 * h)) / (12 * h * h)


def critical_point(eos, a, b, R, K=1.0):
    """(T_c, rho_c) of the oracle's EOS: rho_c(T) is the inflection of the isotherm
    (d2p/drho2 = 0) and T_c the temperature at which the slope there vanishes."""
    rho_max = (1.0 / b) if eos == 0 else (4.0 / b)  # vdW: 1 - b rho > 0; CS: eta < 1

    def inflection(T):
        prm = _params(eos, a, b, R, K, T)
        p = lambda r: O.p_eos(prm, r)
        h = 1e-4 * rho_max
        f = lambda r: _d2(p, r, h)
        # the inflection lies between a small density and the one of the densest state
        lo, hi = 0.05 * rho_max, 0.6 * rho_max
        return brentq(f, lo, hi, xtol=1e-14 * rho_max), p, h

    def slope_at_inflection(T):
        rho_i, p, h = inflection(T)
        return _d1(p, rho_i, h)

    # below T_c the slope at the inflection is negative (van der Waals loop), above positive
    T_guess = 8 * a / (27 * R * b) if eos == 0 else 0.38 * a / (b * R)
    T_c = brentq(slope_at_inflection, 0.7 * T_guess, 1.3 * T_guess, xtol=1e-13 * T_guess)
    rho_c = inflection(T_c)[0]
    return T_c, rho_c


@pytest.mark.parametrize("a,b,K", [(9.0 / 49.0, 2.0 / 21.0, 1.0 / 16.0), (1.0, 0.5, 1.0), (0.3, 0.2, 2.0)])
def test_van_der_waals_critical_point(a, b, K):
    """Sec. 3: T_cr = 8a/(27 R b), rho_cr = 1/(3b) (the paper's a = 9/49, b = 2/21,
    K_EOS = 1/16 first); K_EOS scales the pressure and leaves the critical point."""
    R = 1.0
    T_c, rho_c = critical_point(0, a, b, R, K)
    assert T_c == pytest.approx(8 * a / (27 * R * b), rel=1e-7)
    assert rho_c == pytest.approx(1.0 / (3 * b), rel=1e-6)


@pytest.mark.parametrize("a,b,R", [(1.0, 4.0, 1.0), (0.5, 2.0, 1.0), (2.0, 1.0, 0.5)])
def test_carnahan_starling_critical_point(a, b, R):
    """T_c b R / a = 0.3773 and eta_c = b rho_c / 4 = 0.1304 to four digits (a = 1,
    b = 4, R = 1 is the EOS of every Carnahan-Starling workload here), and the same
    values from oracle/analytic.py's cs_critical."""
    from oracle import analytic as A
    T_c, rho_c = critical_point(1, a, b, R)
    assert round(T_c * b * R / a, 4) == 0.3773, T_c * b * R / a
    assert round(b * rho_c / 4.0, 4) == 0.1304, b * rho_c / 4.0
    Tc_tab, rhoc_tab = A.cs_critical(a, b, R)
    assert Tc_tab == pytest.approx(T_c, rel=2e-4) and rhoc_tab == pytest.approx(rho_c, rel=5e-4)
    # the compressibility factor at the critical point, p_c/(rho_c R T_c) = 0.3590 for CS
    prm = _params(1, a, b, R, 1.0, T_c)
    Z = O.p_eos(prm, rho_c) / (rho_c * R * T_c)
    assert round(Z, 4) == 0.3590, Z


def test_carnahan_starling_hard_sphere_limit():
    """With a = 0 the CS EOS is the hard-sphere compressibility
    Z = (1 + eta + eta^2 - eta^3)/(1 - eta)^3, which at eta = 1/2 is 1.625/0.125 = 13
    and whose virial series starts 1 + 4 eta + 10 eta^2 (second and third virial
    coefficients of hard spheres in units of eta)."""
    b, R, T = 4.0, 1.0, 0.25
    prm = _params(1, 0.0, b, R, 1.0, T)
    rho = 0.5 * 4.0 / b  # eta = 1/2
    assert O.p_eos(prm, rho) / (rho * R * T) == pytest.approx(13.0, rel=1e-14)
    eta = 1e-3
    rho = eta * 4.0 / b
    Z = O.p_eos(prm, rho) / (rho * R * T)
    assert (Z - 1.0 - 4 * eta) / eta ** 2 == pytest.approx(10.0, rel=2e-3)


def test_psi_is_the_eos_inversion():
    """Sec. 2: psi = sqrt(2 (p_EOS - rho/3)/G): rho/3 + G psi^2/2 reproduces p_EOS."""
    prm = _params(1, 1.0, 4.0, 1.0, 1.0, 0.7 * 0.3773 / 4.0)
    prm.G = -1.0
    for rho in (0.01, 0.1, 0.3):
        psi = O.psi(prm, rho)
        assert rho / 3.0 + prm.G * psi * psi / 2.0 == pytest.approx(O.p_eos(prm, rho), rel=1e-12)
        assert math.isfinite(psi) and psi > 0
