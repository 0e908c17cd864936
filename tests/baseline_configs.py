"""The benchmark's named configurations C2-C4 at their stated sizes and lengths, on the GPU
library, each checked against the FP64 oracle over a prefix of the run (the full runs take
the oracle hours).  Prints one JSON line per configuration.

* C2, grid-oblique two-phase Poiseuille flow (Sec. 3.1), 512 x 512, periodic, viscosity
  ratio 10 (tau_l = 1.0, tau_g = 0.55), Carnahan-Starling at 0.7 T_c, 200k steps, FP64 and
  FP32, original vs improved.  A slab at 30 degrees is not periodic on a square lattice, so
  the channel is the paper's 45-degree one: two-node solid bands where (x - y) mod 512 < 2,
  force along the bands.  The channel is 362 nodes wide and its gas layers (nu_g = 1/60)
  accelerate without bound for a long time: the plug's time constant is about 1e7 steps, and
  a force of 1e-7 (C1's) takes the gas to |u| = 0.55 by step 200k, far outside the low-Mach
  regime.  The force is therefore 4e-9 (max |u| about 0.02 at 200k steps); --force changes it.
  Reported: the spurious velocity normal to the bands (max |u_alpha|, zero in the exact
  flow) and its ratio to the velocity along them, Err of the velocity along the bands against
  Eq. (u.plane) integrated with the run's own density (a transient, so not small), FP32
  against FP64.
* C3, annular shear flow (Sec. 3.2), 1024 x 1024: resting inner cylinder r < 128, outer
  cylinder r > 480 moving tangentially at u_w = 0.01, both through interpolated (Bouzidi)
  links; liquid annulus 200 < r < 320 in gas; 500k steps; FP32 against FP16 (rounded to
  nearest and stochastically) and BF16 deviation storage (per-node reference).  The run proceeds in chunks and records the first
  chunk that ends with a non-finite field: interpolated bounce-back does not conserve mass
  where the wall holds a density gradient (the adsorbed gas layer), and the heavy ring
  between lighter gas is the Rayleigh-Taylor-unstable layout that Sec. 3.2 avoids.  The
  same geometry with half-way walls on the staircase of solid nodes runs beside it.
* C4, droplet falling in a vertical channel (Sec. 3.3), 512 x 4096, half-way side walls,
  periodic top and bottom; droplet of radius 40 at a seed-4 jittered centre near (256, 3500)
  in gas at the density in equilibrium with it (see _vapour_density; in Maxwell gas the
  droplet evaporates within 40k steps); relaxed without gravity, then buoyant gravity
  (rho - rho_g) g with |g| = 2e-6, rho_g that ambient density; 300k steps; original and
  improved scheme, FP32 and FP16 (rounded to nearest and stochastically); FP64 reductions of mass, the momentum handed to the walls
  (drag) and U_c, and the droplet's equivalent radius and centre line.

    python -m tests.baseline_configs [--configs c2,c3,c4] [--scale S] [--prefix P] [--force F]

--scale divides the step counts (for a quick look); --prefix is the length of the oracle
comparison.
"""
import argparse
import json
import math
import time

import numpy as np

from oracle import analytic as A
from oracle import oracle as O
from paper_2604_13407_gb300 import inputs as I
from tests import gpu_cases as GC
from tests.setups import cs_case, cs_params


def _field_err(sim, ref, solid=None):
    """(max |du| / max |u_ref|, max relative rho error) over fluid nodes; ref is a
    Simulation or an OracleSim."""
    return GC.field_errors(sim, ref, solid)[::-1]


def _glups(sim, n_nodes, steps):
    """Lattice updates per second over `steps` steps, host clock between two
    synchronisations of the simulation's own stream (launches are asynchronous, so the
    interval is the device time of the steps plus one launch latency)."""
    sim.sync()
    t0 = time.perf_counter()
    sim.step(steps)
    sim.sync()
    return n_nodes * steps / (time.perf_counter() - t0) / 1e9


def _oracle_prefix(case, steps):
    o = GC.run_oracle(case, steps=steps)
    return o


# ---------------------------------------------------------------------- C2 ----
def _c2_series(s, steps, fluid, chunks=8):
    """Step in `chunks` chunks; after each, the largest velocity along the bands and normal
    to them over fluid nodes."""
    rows = []
    for k in range(chunks):
        s.step(steps // chunks)
        rho, ux, uy = s.moments()
        ua = np.abs(ux - uy)[fluid] / math.sqrt(2)
        ub = np.abs(ux + uy)[fluid] / math.sqrt(2)
        rows.append({"step": (k + 1) * (steps // chunks), "max_u_along": float(ub.max()),
                     "normal_max": float(ua.max()), "normal_rms": float(np.sqrt((ua * ua).mean()))})
    return rows


def c2(lbm, steps=200000, prefix=2000, n=512, F=4e-9):
    T, rg, rl = cs_case()
    solid = I.oblique_band_walls(n)
    rho0 = np.where(solid == 1, rg, I.oblique_slab(n, rl, rg, n // 2))
    fluid = solid == 0
    out = {"config": "C2", "lattice": "%dx%d" % (n, n), "steps": steps,
           "geometry": "45-degree channel, two-node solid bands where (x - y) mod %d < 2" % n,
           "force": F, "tau_l": 1.0, "tau_g": 0.55, "schemes": {}}
    nu_fn = lambda r: A.nu_of_rho(r, 1.0, 0.55, rl, rg)
    idx = np.arange(2, n)
    for scheme in (0, 1):
        p = cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True, Fx=F / math.sqrt(2), Fy=F / math.sqrt(2),
                      tau_l=1.0, tau_g=0.55, scheme=scheme)
        case = GC.Case("c2", p, rho0, steps, solid=solid)
        res = {}
        # oracle prefix
        o = _oracle_prefix(case, prefix)
        for prec, name in ((lbm.F64, "f64"), (lbm.F32, "f32")):
            g = GC.run_gpu(case, prec, steps=prefix)
            eu, er = _field_err(g, o, solid)
            res["%s_vs_oracle_%d_steps" % (name, prefix)] = {"e_u": eu, "e_rho": er}
        # full runs (FP32 in chunks, with the spurious normal velocity after each)
        sims = {}
        for prec, name in ((lbm.F64, "f64"), (lbm.F32, "f32")):
            t0 = time.time()
            if prec == lbm.F32:
                s = GC.run_gpu(case, prec, steps=0)
                res["f32_series"] = _c2_series(s, steps, fluid)
            else:
                s = GC.run_gpu(case, prec)
            s.sync()
            res[name + "_seconds"] = round(time.time() - t0, 1)
            res[name + "_kernel"] = ["auto", "two_pass", "fused"][s.kernel_in_use]
            sims[name] = s
        # the same channel with one relaxation time (tau = 1 in both phases), FP32
        pu = cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True, Fx=F / math.sqrt(2), Fy=F / math.sqrt(2),
                       tau_l=1.0, tau_g=1.0, scheme=scheme)
        su = GC.run_gpu(GC.Case("c2u", pu, rho0, steps, solid=solid), lbm.F32, steps=0)
        res["f32_tau1_series"] = _c2_series(su, steps, fluid)
        su.close()
        eu, er = _field_err(sims["f32"], sims["f64"], solid)
        res["f32_vs_f64_full"] = {"e_u": eu, "e_rho": er}
        for name, s in sims.items():
            rho, ux, uy = s.moments()
            ua = (ux - uy) / math.sqrt(2)
            ub = (ux + uy) / math.sqrt(2)
            th = A.poiseuille_theory(rho[0, idx], F, nu_fn, spacing=1.0 / math.sqrt(2))
            res[name + "_flow"] = {
                "max_u_along": float(np.abs(ub[fluid]).max()),
                "spurious_normal_max": float(np.abs(ua[fluid]).max()),
                "spurious_normal_rel": float(np.abs(ua[fluid]).max() / np.abs(ub[fluid]).max()),
                "Err_vs_u_plane": A.err_norm((ux[0, idx] + uy[0, idx]) / math.sqrt(2), th),
                "density_ratio": float(rho[0, idx].max() / rho[0, idx].min())}
        res["glups_f32"] = _glups(sims["f32"], int(fluid.size), 2000)
        res["glups_f64"] = _glups(sims["f64"], int(fluid.size), 200)
        out["schemes"]["original" if scheme == 0 else "improved"] = res
        for s in sims.values():
            s.close()
    return out


# ---------------------------------------------------------------------- C3 ----
def _run_chunked(s, steps, chunk, fluid, m0, keep_at=None):
    """Step a simulation in chunks, recording mass drift and max |u| after each; stops at
    the first chunk whose diagnostics report a non-finite field.  Returns (rows, step of
    the blow-up or None, moments at step keep_at or None)."""
    from paper_2604_13407_gb300 import lbm
    rows, kept = [], None
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        s.step(k)
        done += k
        try:
            d = s.diagnostics()
        except lbm.LbmError as e:
            if lbm.STATUS.get(e.status) != "LBM_ENAN":
                raise
            return rows, done, kept
        rho, ux, uy = s.moments()
        rows.append({"step": done, "mass_drift": d[0] / m0 - 1.0,
                     "max_u": float(np.hypot(ux, uy)[fluid].max())})
        if keep_at is not None and done == keep_at:
            kept = (rho, ux, uy)
    return rows, None, kept


def _moment_err(a, b, fluid):
    """(max |du| / max |u_b|, max relative rho error) between two moment triples."""
    umax = max(np.abs(b[1][fluid]).max(), np.abs(b[2][fluid]).max())
    eu = max(np.abs(a[1] - b[1])[fluid].max(), np.abs(a[2] - b[2])[fluid].max()) / umax
    er = float((np.abs(a[0] - b[0]) / np.abs(b[0]))[fluid].max())
    return float(eu), er


def c3(lbm, steps=500000, prefix=2000, n=1024, chunk=25000, compare_at=25000):
    T, rg, rl = cs_case()
    solid, wall_u, q = I.annulus(n, n, 128.0, 480.0, u_wall_out=0.01)
    c0 = (n - 1) / 2
    r = np.hypot(np.arange(n)[None, :] - c0, np.arange(n)[:, None] - c0)
    ring = rg + 0.5 * (rl - rg) * (np.tanh(2 * (r - 200.0) / 4.0) - np.tanh(2 * (r - 320.0) / 4.0))
    rho0 = np.where(solid == 1, rg, ring)
    fluid = solid == 0
    p = cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True, scheme=1)
    case = GC.Case("c3", p, rho0, steps, solid=solid, wall_u=wall_u, q=q)
    out = {"config": "C3", "lattice": "%dx%d" % (n, n), "steps": steps, "chunk": chunk,
           "geometry": "resting cylinder r < 128, cylinder r > 480 moving at 0.01, interpolated links; "
                       "liquid annulus 200 < r < 320"}
    precs = (("f32", lbm.F32, {}), ("f16dev_nearest", lbm.F16DEV, {"per_node_ref": 1, "storage_rounding": 0}),
             ("f16dev_stochastic", lbm.F16DEV, {"per_node_ref": 1, "storage_rounding": 1}),
             ("bf16dev_stochastic", lbm.BF16DEV, {"per_node_ref": 1, "storage_rounding": 1}))
    o = _oracle_prefix(case, prefix)
    out["oracle_mass_drift_%d_steps" % prefix] = float(o.moments()[0][fluid].sum() / rho0[fluid].sum() - 1.0)
    for name, prec, kw in precs:
        g = GC.run_gpu(case, prec, steps=prefix, **kw)
        eu, er = _field_err(g, o, solid)
        out["%s_vs_oracle_%d_steps" % (name, prefix)] = {"e_u": eu, "e_rho": er, "kernel": ["auto", "two_pass", "fused"][g.kernel_in_use]}
        out["%s_mass_drift_%d_steps" % (name, prefix)] = float(g.moments()[0][fluid].sum() / rho0[fluid].sum() - 1.0)
        g.close()
    kept = {}
    runs = precs + (("f32_halfway", lbm.F32, {}),)
    for name, prec, kw in runs:
        t0 = time.time()
        c = case if name != "f32_halfway" else GC.Case("c3h", p, rho0, steps, solid=solid, wall_u=wall_u)
        s = GC.run_gpu(c, prec, steps=0, **kw)
        m0 = s.diagnostics()[0]
        rows, blew, kept[name] = _run_chunked(s, steps, chunk, fluid, m0, keep_at=compare_at)
        out[name] = {"seconds": round(time.time() - t0, 1), "series": rows, "non_finite_at": blew}
        if blew is None:
            out[name]["glups"] = _glups(s, int(fluid.size), 2000)
        s.close()
    for name in ("f16dev_nearest", "f16dev_stochastic", "bf16dev_stochastic"):
        if kept[name] is not None and kept["f32"] is not None:
            eu, er = _moment_err(kept[name], kept["f32"], fluid)
            out["%s_vs_f32_%d_steps" % (name, compare_at)] = {"e_u": eu, "e_rho": er}
    return out


# ---------------------------------------------------------------------- C4 ----
def _vapour_density(lbm, radius, steps=20000):
    """Gas density in equilibrium with a droplet of this radius: a droplet centred in a
    periodic 4R x 4R box relaxed for `steps` steps (FP64 on the GPU), read at the corner.
    At 0.7 T_c it is 22 % above the Maxwell gas density for R = 40 (the Laplace pressure of
    the curved interface), so a droplet started in Maxwell gas evaporates into a large
    channel: 512 x 4096 nodes of gas take up that 22 % with more mass than the droplet has."""
    T, rg, rl = cs_case()
    n = int(4 * radius)
    p = cs_params(nx=n, ny=n, periodic_x=True, periodic_y=True, scheme=1)
    rho0 = I.droplet(n, n, rl, rg, radius, (n - 1) / 2, (n - 1) / 2, periodic_x=True, periodic_y=True)
    s = GC.run_gpu(GC.Case("vap", p, rho0, steps), lbm.F64)
    rv = float(s.moments()[0][0, 0])
    s.close()
    return rv


def c4(lbm, steps=300000, prefix=1000, relax=20000, nx=512, ny=4096, g=2e-6, radius=40.0, samples=15):
    T, rg, rl = cs_case()
    rv = _vapour_density(lbm, radius)
    cx, cy = I.jittered_centre(4, 256.0, 3500.0)
    rho0 = I.droplet(nx, ny, rl, rv, radius, cx, cy, periodic_x=False, periodic_y=True)
    # the ambient gas density is the buoyancy reference, (rho - rho_g) g, and the walls'
    mk = lambda gy, scheme: cs_params(nx=nx, ny=ny, periodic_x=False, periodic_y=True, force_mode=1, Fy=gy,
                                      scheme=scheme, rho_g=rv, rho_s=rv)
    out = {"config": "C4", "lattice": "%dx%d" % (nx, ny), "steps": steps, "relax_steps": relax,
           "droplet": {"radius": radius, "centre": [cx, cy]}, "gravity": g,
           "gas_density": {"maxwell": rg, "with_droplet": rv}}
    # the oracle prefix, with gravity from the start
    case = GC.Case("c4", mk(-g, 1), rho0, prefix)
    o = _oracle_prefix(case, prefix)
    c4_precs = (("f32", lbm.F32, {}), ("f16dev_nearest", lbm.F16DEV, {"per_node_ref": 1, "storage_rounding": 0}),
                ("f16dev_stochastic", lbm.F16DEV, {"per_node_ref": 1, "storage_rounding": 1}))
    for name, prec, kw in c4_precs:
        s = GC.run_gpu(case, prec, **kw)
        eu, er = _field_err(s, o)
        out["%s_vs_oracle_%d_steps" % (name, prefix)] = {"e_u": eu, "e_rho": er, "kernel": ["auto", "two_pass", "fused"][s.kernel_in_use]}
        s.close()
    series = {}
    xs = np.arange(nx)[None, :]
    ys = np.arange(ny)[:, None]
    for scheme in (0, 1):
        for name, prec, kw in c4_precs:
            key = "%s_%s" % ("original" if scheme == 0 else "improved", name)
            t0 = time.time()
            s = lbm.Simulation(GC.gpu_params(mk(0.0, scheme), prec, **kw))
            s.init_fields(rho0)
            s.step(relax)
            s.set_param(lbm.PARAM_FY, -g)
            m0 = s.diagnostics()[0]
            rows = []
            chunk = steps // samples
            for k in range(samples):
                s.step(chunk)
                d = s.diagnostics()
                rho, ux, uy = s.moments()
                liquid = rho > 0.5 * (rl + rv)
                nl = int(liquid.sum())
                # d[4]: total y force on the fluid (buoyancy; the pairwise force sums to zero);
                # d[6]: y momentum handed to the walls by the last streaming (drag); d[7]/d[8]: U_c
                row = {"step": (k + 1) * chunk, "U_c": d[7] / d[8] if d[8] > 0 else None, "drag_y": d[6],
                       "force_y": d[4], "mass_drift": d[0] / m0 - 1.0, "R_eq": math.sqrt(nl / math.pi)}
                if nl:
                    row["centre_x"] = float((xs * liquid).sum() / nl)
                rows.append(row)
            out[key + "_seconds"] = round(time.time() - t0, 1)
            out[key + "_glups"] = _glups(s, nx * ny, 2000)
            series[key] = rows
            s.close()
    out["series"] = series
    for key, rows in series.items():
        last = rows[-1]
        if last["U_c"] is None:
            continue
        # quasi-steady fall: the walls take up the buoyancy, sum F = D (momentum balance)
        out[key + "_momentum_balance"] = abs(last["drag_y"] - last["force_y"]) / abs(last["force_y"])
        out[key + "_U_c"] = last["U_c"]
    for sch in ("original", "improved"):
        for name in ("f16dev_nearest", "f16dev_stochastic"):
            a, b = out.get("%s_%s_U_c" % (sch, name)), out.get(sch + "_f32_U_c")
            if a is not None and b is not None:
                out["%s_%s_vs_f32_U_c" % (sch, name)] = abs(a - b) / abs(b)
    return out


def main():
    import torch
    from paper_2604_13407_gb300 import lbm
    ap = argparse.ArgumentParser()
    ap.add_argument("--configs", default="c2,c3,c4")
    ap.add_argument("--scale", type=int, default=1, help="divide the step counts by this")
    ap.add_argument("--prefix", type=int, default=None, help="oracle prefix length (steps)")
    ap.add_argument("--force", type=float, default=None, help="C2's driving force")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    runs = {"c2": (c2, 200000), "c3": (c3, 500000), "c4": (c4, 300000)}
    for name in args.configs.split(","):
        fn, steps = runs[name]
        kw = {"steps": steps // args.scale}
        if args.prefix:
            kw["prefix"] = args.prefix
        if name == "c4" and args.scale > 1:
            kw["relax"] = 20000 // args.scale
        if name == "c3" and args.scale > 1:
            kw["chunk"] = kw["compare_at"] = 25000 // args.scale
        if name == "c2" and args.force is not None:
            kw["F"] = args.force
        t0 = time.time()
        res = fn(lbm, **kw)
        res["wall_seconds"] = round(time.time() - t0, 1)
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
