"""Seeded cases run on both the CUDA library and the FP64 oracle (tests only)."""
import dataclasses
import math

import numpy as np

from oracle import oracle as O
from paper_2604_13407_gb300 import inputs as I
from paper_2604_13407_gb300 import lbm
from tests.setups import cs_case, cs_params

SHARED = ["nx", "ny", "periodic_x", "periodic_y", "scheme", "q2_original", "eos", "force_mode",
          "a", "b", "R", "T", "K_eos", "G", "k1", "k2", "tau_l", "tau_g", "rho_l", "rho_g",
          "Lambda", "Fx", "Fy", "rho_s"]


@dataclasses.dataclass
class Case:
    name: str
    params: O.Params
    rho0: np.ndarray
    steps: int
    solid: np.ndarray = None
    wall_u: np.ndarray = None
    q: np.ndarray = None
    fext: np.ndarray = None


# FP16 deviation storage scales 2^k keeping |f_i - w_i rho_ref| 2^k in the normal FP16
# range: deviations from the node's own density stay well below 0.25, those from a global
# reference below ~0.2 (w_0 (rho_l - rho_g)).
HALF_SCALE = {True: 18, False: 17}


def gpu_params(op: O.Params, precision, kernel=lbm.KERNEL_AUTO, **kw):
    p = lbm.default_params()
    for f in SHARED:
        v = getattr(op, f)
        setattr(p, f, int(v) if isinstance(v, bool) else v)
    p.precision = precision
    p.kernel = kernel
    p.rho_ref = op.rho_g
    if precision == lbm.F16DEV:
        p.storage_scale_log2 = HALF_SCALE[bool(kw.get("per_node_ref", 0))]
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def run_gpu(case: Case, precision, kernel=lbm.KERNEL_AUTO, steps=None, **kw):
    sim = lbm.Simulation(gpu_params(case.params, precision, kernel, **kw))
    if any(a is not None for a in (case.solid, case.wall_u, case.q, case.fext)):
        sim.set_geometry(case.solid, case.wall_u, case.q, case.fext)
    sim.init_fields(case.rho0)
    sim.step(case.steps if steps is None else steps)
    return sim


def run_oracle(case: Case, steps=None):
    s = O.OracleSim(case.params, solid=case.solid, wall_u=case.wall_u, q=case.q, fext=case.fext)
    s.init(case.rho0)
    s.step(case.steps if steps is None else steps)
    return s


def cases():
    T, rg, rl = cs_case()
    out = {}
    for scheme in (0, 1):
        p = cs_params(nx=4, ny=64, periodic_x=True, periodic_y=False, Fx=1e-6, scheme=scheme)
        out["channel_s%d" % scheme] = Case("channel_s%d" % scheme, p, I.tanh_slab(4, 64, rl, rg, 32), 3000)
    p = cs_params(nx=40, ny=48, periodic_x=True, periodic_y=True, force_mode=1, Fy=-2e-5, scheme=1)
    out["droplet"] = Case("droplet", p, I.droplet(40, 48, rl, rg, 9, 19.3, 25.1, periodic_x=True), 400)
    n = 32
    f = 1e-6
    p = cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True, Fx=f / math.sqrt(2), Fy=f / math.sqrt(2),
                  tau_l=1.0, tau_g=0.55, scheme=1)
    out["oblique"] = Case("oblique", p, I.oblique_slab(n, rl, rg, 14), 500, solid=I.oblique_band_walls(n))
    n = 64
    solid, wall_u, q = I.annulus(n, n, 8.3, 29.6, u_wall_out=0.01)
    c0 = (n - 1) / 2
    r = np.hypot(np.arange(n)[None, :] - c0, np.arange(n)[:, None] - c0)
    ring = rg + 0.5 * (rl - rg) * (np.tanh(2 * (r - 14.0) / 4.0) - np.tanh(2 * (r - 22.0) / 4.0))
    p = cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True, scheme=1)
    out["annulus"] = Case("annulus", p, np.where(solid == 1, rg, ring), 250, solid=solid, wall_u=wall_u, q=q)
    p = cs_params(nx=37, ny=23, periodic_x=True, periodic_y=False, Fx=3e-6, Fy=1e-6, scheme=0)
    out["ragged"] = Case("ragged", p, I.droplet(37, 23, rl, rg, 6, 17.2, 11.0, periodic_x=True), 250)
    p = cs_params(nx=1, ny=5, periodic_x=True, periodic_y=True, scheme=1)
    out["tiny"] = Case("tiny", p, (0.15 + 0.05 * np.sin(2 * np.pi * np.arange(5) / 5)).reshape(5, 1), 50)
    return out


def field_errors(sim, oracle_sim, solid=None):
    """(max relative rho error, max |du| / max |u|) over fluid nodes."""
    rg, ug, vg = sim.moments()
    ro, uo, vo = oracle_sim.moments()
    fluid = np.ones_like(ro, dtype=bool) if solid is None else (solid == 0)
    e_rho = np.max(np.abs(rg - ro)[fluid] / np.abs(ro)[fluid])
    umax = max(np.abs(uo[fluid]).max(), np.abs(vo[fluid]).max(), 1e-300)
    e_u = max(np.abs(ug - uo)[fluid].max(), np.abs(vg - vo)[fluid].max()) / umax
    return e_rho, e_u
