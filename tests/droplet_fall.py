"""Droplet falling in a vertical channel, Sec. 3.3, on the GPU library, with half-way
bounce-back walls and the virtual wall density rho_s = rho_g in place of the paper's wall
scheme.

Set-up (Sec. 3.3): van der Waals EOS (a = 9/49, b = 2/21, R = 1, K_EOS = 1/16) at
T_r = 0.5 (liquid-to-gas ratio about 113), epsilon = 1.895 (k1 = k2 = -epsilon/16),
tau = 0.8, Lambda = 1/12; channel W = 256 wide (walls at x = -1/2 and 255.5), H = 2048
high and periodic in y; a droplet of diameter D = 128 centred in the channel.  The run is
first relaxed without gravity, then the buoyant gravity (rho - rho_g) g, |g| in
{0.5, 1, 2} x 1e-7, pulls it down.  Recorded along the fall: the falling velocity
U_c = int rho u_y dA / int rho dA over the liquid region (rho above the mean of the
coexistence densities) and its reduced forms U_c* = U_c / sqrt(|g| D (rho_l - rho_g)/rho_g),
t* = t / sqrt(D/|g|), and the centre of mass of the liquid across the channel (the
migration towards a wall).  Nothing seeds the symmetry breaking but rounding, as in the
paper.

Run as `python -m tests.droplet_fall [--precision f32|f64] [--t-max 300]` (JSON lines: one
per sample and a summary per run).
"""
import argparse
import json
import math
import sys
import time

import numpy as np

from paper_2604_13407_gb300 import inputs as I
from tests.setups import vdw_case, vdw_params
from tests.table1 import psi_real_limit

W, H, D = 256, 2048, 128.0
T_R, EPS, TAU = 0.5, 1.895, 0.8
GRAVITIES = (0.5e-7, 1.0e-7, 2.0e-7)
RELAX_STEPS = 60000

# Sec. 3.3: terminal |U_c*| (original, improved) per |g|, and the migration onset
PAPER_TERMINAL = {0.5e-7: (0.9144, 1.0104), 1.0e-7: (1.2535, 0.9015), 2.0e-7: (1.1116, 1.0928)}
PAPER_ONSET_2E7 = {"t_star": (107.6, 53.8), "U_c_star": 1.92}


def make_sim(lbm, scheme, precision, g, kernel=0):
    from tests import gpu_cases as GC
    T, rg, rl = vdw_case(T_R)
    op = vdw_params(EPS, T_R, nx=W, ny=H, periodic_x=False, periodic_y=True, force_mode=1,
                    Fx=0.0, Fy=-g, scheme=scheme, tau_l=TAU, tau_g=TAU)
    gp = GC.gpu_params(op, precision, kernel)
    gp.rho_max = psi_real_limit(op, rl)
    return lbm.Simulation(gp)


def liquid_centre_x(rho, rho_cut):
    w = np.where(rho > rho_cut, rho, 0.0)
    return float((w.sum(axis=0) * np.arange(W)).sum() / w.sum())


def run(lbm, scheme, g, precision, t_max, sample_every=1.0, relaxed=None, kernel=0):
    """Relax without gravity (or start from `relaxed`), then fall; yields sample dicts and
    returns the relaxed state for reuse by the next |g| of the same scheme."""
    T, rg, rl = vdw_case(T_R)
    rho_cut = 0.5 * (rl + rg)
    sim = make_sim(lbm, scheme, precision, 0.0, kernel)
    if relaxed is None:
        sim.init_fields(I.droplet(W, H, rl, rg, D / 2.0, (W - 1) / 2.0, H / 2.0, periodic_x=False, periodic_y=True))
        sim.step(RELAX_STEPS)
        relaxed = sim.get_state()
    else:
        sim.set_state(relaxed)
    sim.set_param(lbm.PARAM_FY, -g)
    sim.sync()
    t_fall = time.time()
    t_unit = math.sqrt(D / g)
    u_unit = math.sqrt(g * D * (rl - rg) / rg)
    samples = []
    t_done = 0
    k = 0
    while True:
        k += 1
        target = int(round(k * sample_every * t_unit))
        if target * 1.0 / t_unit > t_max + 1e-9:
            break
        sim.step(target - t_done)
        t_done = target
        d = sim.diagnostics()
        rho, _, _ = sim.moments()
        s = {"t_star": t_done / t_unit, "U_c_star": d[7] / d[8] / u_unit,
             "x_c_over_W": (liquid_centre_x(rho, rho_cut) + 0.5) / W, "max_u": d[9]}
        if not np.isfinite(s["U_c_star"]):
            raise RuntimeError("non-finite state at t* = %.1f" % s["t_star"])
        samples.append(s)
    run.us_per_step = 1e6 * (time.time() - t_fall) / max(t_done, 1)
    return samples, relaxed


def summarise(samples, scheme, g):
    t = np.array([s["t_star"] for s in samples])
    u = np.abs(np.array([s["U_c_star"] for s in samples]))
    xc = np.array([s["x_c_over_W"] for s in samples])
    tail = t >= 0.85 * t[-1]
    off = np.nonzero(np.abs(xc - 0.5) > 0.05)[0]
    onset = None if len(off) == 0 else int(off[0])
    # the onset of migration: the last sample within 1 % of the centre line before leaving 5 %
    start = None
    if onset is not None:
        near = np.nonzero(np.abs(xc[:onset] - 0.5) < 0.01)[0]
        start = int(near[-1]) if len(near) else 0
    return {"summary": True, "scheme": ["original", "improved"][scheme], "g": g,
            "terminal_U_c_star": float(u[tail].mean()), "terminal_spread": float(u[tail].std()),
            "final_x_c_over_W": float(xc[-1]),
            "migration_t_star": None if start is None else float(t[start]),
            "U_c_star_at_migration": None if start is None else float(u[start]),
            "paper_terminal_U_c_star": PAPER_TERMINAL[g][scheme]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", choices=("f32", "f64"), default="f32")
    ap.add_argument("--t-max", type=float, default=300.0)
    ap.add_argument("--g", type=float, nargs="*", default=list(GRAVITIES))
    ap.add_argument("--scheme", type=int, nargs="*", default=[0, 1])
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 two-pass, 2 fused")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    from paper_2604_13407_gb300 import lbm
    precision = {"f32": lbm.F32, "f64": lbm.F64}[args.precision]
    for scheme in args.scheme:
        relaxed = None
        for g in args.g:
            t0 = time.time()
            samples, relaxed = run(lbm, scheme, g, precision, args.t_max, relaxed=relaxed, kernel=args.kernel)
            for s in samples:
                print(json.dumps(dict(s, scheme=scheme, g=g)))
            out = summarise(samples, scheme, g)
            out["seconds"] = round(time.time() - t0, 1)
            out["us_per_step_falling"] = round(run.us_per_step, 2)
            out["kernel_in_use"] = args.kernel
            print(json.dumps(out), flush=True)


if __name__ == "__main__":
    sys.exit(main())
