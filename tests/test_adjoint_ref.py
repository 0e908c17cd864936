"""Pins of the FP64 reference adjoint (oracle/adjoint_ref.py): its forward pass equals the
C oracle, its gradients equal central finite differences of the C oracle, dJ/dG = 0
(G drops out of the method, Sec. 2), and a single-phase channel's mean flux is linear in
the force."""
import dataclasses

import numpy as np
import pytest

from oracle import adjoint_ref as AR
from oracle import oracle as O
from paper_2604_13407_gb300 import inputs as I
from tests.setups import cs_case, cs_params


def channel_case():
    T, rg, rl = cs_case()
    p = cs_params(nx=6, ny=20, periodic_x=True, periodic_y=False, Fx=2e-6, scheme=1, tau_l=0.9, tau_g=0.7)
    return p, I.tanh_slab(6, 20, rl, rg, 10), None


def droplet_case():
    T, rg, rl = cs_case()
    p = cs_params(nx=14, ny=16, periodic_x=False, periodic_y=True, force_mode=1, Fx=1e-6, Fy=-3e-6, scheme=0)
    solid = np.zeros((16, 14), np.uint8)
    solid[5:7, 9:11] = 1
    rho = I.droplet(14, 16, rl, rg, 3.5, 5.6, 8.3, periodic_x=False, periodic_y=True)
    return p, np.where(solid == 1, rg, rho), solid


def initial_state(p, rho, solid):
    s = O.OracleSim(p, solid=solid)
    s.init(rho)
    return s.get_state()


def oracle_J(p, A0, n, objective, solid):
    s = O.OracleSim(p, solid=solid)
    s.set_state(A0)
    states = []
    for _ in range(n):
        s.step(1)
        states.append(s.get_state())
    return AR.objective_value(p, states, objective, solid)


@pytest.mark.parametrize("case", [channel_case, droplet_case])
def test_reference_forward_equals_oracle(case):
    p, rho, solid = case()
    A0 = initial_state(p, rho, solid)
    ref = AR.forward_states(p, A0, 15, solid)
    s = O.OracleSim(p, solid=solid)
    s.set_state(A0)
    fluid = np.ones((p.ny, p.nx), bool) if solid is None else solid == 0
    for t in range(15):
        s.step(1)
        assert np.abs(ref[t] - s.get_state())[:, fluid].max() < 1e-14


@pytest.mark.parametrize("case,objective", [(channel_case, "mean_jx"), (droplet_case, "wall_force_y"),
                                            (droplet_case, "mean_jx")])
def test_reference_gradient_equals_finite_differences(case, objective):
    p, rho, solid = case()
    A0 = initial_state(p, rho, solid)
    n = 12
    J, g, lam = AR.objective_and_grad(p, A0, n, objective, solid)
    # J is a sum of O(1e-3) terms that cancel down to O(1e-5): compare at 1e-11 relative
    assert abs(J - oracle_J(p, A0, n, objective, solid)) <= 1e-11 * max(abs(J), 1e-30)
    for k, name in ((0, "Fx"), (1, "Fy"), (3, "T")):
        v = getattr(p, name)
        h = 1e-4 * abs(v) if v != 0 else 1e-7
        Jp = oracle_J(dataclasses.replace(p, **{name: v + h}), A0, n, objective, solid)
        Jm = oracle_J(dataclasses.replace(p, **{name: v - h}), A0, n, objective, solid)
        fd = (Jp - Jm) / (2 * h)
        assert abs(g[k] - fd) <= 1e-5 * max(abs(fd), abs(g[k])) + 1e-12 * abs(J) / h, (name, g[k], fd)
    # dJ/dA0 along a random direction
    rng = np.random.default_rng(3)
    d = rng.normal(size=A0.shape) * 1e-3 * np.abs(A0).max()
    if solid is not None:
        d[:, solid == 1] = 0.0
    eps = 1e-4
    fd = (oracle_J(p, A0 + eps * d, n, objective, solid) - oracle_J(p, A0 - eps * d, n, objective, solid)) / (2 * eps)
    assert abs((lam * d).sum() - fd) <= 1e-6 * abs(fd) + 1e-14


def test_reference_gradient_wrt_G_is_zero():
    p, rho, solid = droplet_case()
    A0 = initial_state(p, rho, solid)
    J, g, _ = AR.objective_and_grad(p, A0, 10, "wall_force_y", solid)
    # G enters psi as |G|^-1/2 and the force and source as G psi psi: the derivative
    # cancels exactly, so what remains is round-off of the chain rule
    scale = np.abs(g[[0, 1, 3]]).max() + abs(J)
    assert abs(g[2]) < 1e-10 * scale


def test_single_phase_flux_linear_in_force():
    """Uniform density, walls at rho_s = rho: F_int = 0 and the flow is linear in F up to
    the O(u^2) equilibrium terms, so dJ/dFx = J/Fx to ~1e-6 at these speeds."""
    p = cs_params(nx=4, ny=12, periodic_x=True, periodic_y=False, Fx=1e-6, rho_s=0.3, scheme=1)
    A0 = initial_state(p, np.full((12, 4), 0.3), None)
    J, g, _ = AR.objective_and_grad(p, A0, 30, "mean_jx", None)
    assert abs(g[0] - J / p.Fx) < 1e-6 * abs(J / p.Fx)
