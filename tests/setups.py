"""Shared test set-ups: parameters of the Carnahan-Starling and van der Waals cases and
their coexistence densities, computed by the oracle's analytic module only."""
import functools
import math

from oracle import analytic as A
from oracle import oracle as O

CS = dict(eos=1, a=1.0, b=4.0, R=1.0)
EPS_TC = 1.895  # thermodynamically consistent epsilon of Secs. 3.2-3.3


@functools.lru_cache(maxsize=None)
def cs_case(t_ratio=0.7):
    """(T, rho_g, rho_l) of the Carnahan-Starling EOS at T = t_ratio * T_c (Maxwell)."""
    Tc, _ = A.cs_critical(CS["a"], CS["b"], CS["R"])
    T = t_ratio * Tc
    rg, rl, _ = A.maxwell(1, CS["a"], CS["b"], CS["R"], T)
    return T, rg, rl


@functools.lru_cache(maxsize=None)
def vdw_case(t_r):
    """(T, rho_g, rho_l) of the paper's van der Waals EOS (Sec. 3: a = 9/49, b = 2/21,
    R = 1, K_EOS = 1/16) at reduced temperature t_r (Maxwell densities)."""
    a, b = 9.0 / 49.0, 2.0 / 21.0
    Tc, _ = A.vdw_critical(a, b, 1.0)
    T = t_r * Tc
    rg, rl, _ = A.maxwell(0, a, b, 1.0, T, 1.0 / 16.0)
    return T, rg, rl


def cs_params(eps=EPS_TC, **kw):
    T, rg, rl = cs_case()
    k = -eps / 16.0
    base = dict(eos=1, a=1.0, b=4.0, R=1.0, T=T, K_eos=1.0, G=-1.0, k1=k, k2=k,
                rho_l=rl, rho_g=rg, rho_s=rg)
    base.update(kw)
    return O.Params(**base)


def vdw_params(eps, t_r, **kw):
    T, rg, rl = vdw_case(t_r)
    k = -eps / 16.0
    base = dict(eos=0, a=9.0 / 49.0, b=2.0 / 21.0, R=1.0, T=T, K_eos=1.0 / 16.0, G=-1.0,
                k1=k, k2=k, rho_l=rl, rho_g=rg, rho_s=rg)
    base.update(kw)
    return O.Params(**base)


def s_q(tau, Lambda=1.0 / 12.0):
    """(1/s_q - 1/2)(1/s_p - 1/2) = Lambda with s_p = 1/tau (Sec. 3)."""
    return 1.0 / (0.5 + Lambda / (tau - 0.5))


SQRT2 = math.sqrt(2.0)
