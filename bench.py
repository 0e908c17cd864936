"""Throughput of the D2Q9 pseudopotential MRT step on the periodic spinodal workload.

Workload: 8192 x 8192 periodic lattice, Carnahan-Starling EOS (a = 1, b = 4, R = 1,
T = 0.7 T_c), epsilon = 1.895, improved third-order source, tau = 1.0 (at tau = 0.8 the
spinodal transient reaches |u| ~ 0.26 and is marginally stable), initial density
rho = (rho_l + rho_g)/2 (1 + U(-0.01, 0.01)) with SplitMix64 seed 5, u = 0.  One step is
one lattice update of every node.  Inputs (two 2.4 GB population buffers in FP32) are
far larger than the 129 MB L2, so no flush is needed between steps.

Prints one JSON line.  With --variants (the default) it also times the other storage types
and the original scheme on this workload, and the one-pass step on lattices shaped like the
two-phase channel, annulus and falling-droplet configurations ("geometry").  --impl reference
times the FP64 CPU oracle instead (bounded sample of the same workload on the host cores).
"""
import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RHO_G, RHO_L = 0.009291723294794338, 0.3581443962580134  # Maxwell densities of the EOS at 0.7 T_c
T_07 = 0.7 * 0.3773 / 4.0
TAU = 1.0
BYTES = {"f64": 144, "f32": 72, "f16dev": 36, "bf16dev": 36}
# DRAM bytes per lattice update of the packed fused kernel (k_fused2), from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch at 4096 x 4096; profiles/k_fused2_*;
# f16dev: the per-node reference mode), scaled to a launch by the updates it makes.
# Valid for the kernel as captured; an entry is removed when the kernel changes until it is captured
# again (the line then reports traffic null).
TRAFFIC_PER_UPDATE = {"f32": 73.86, "f16dev": 43.93}
HBM_FALLBACK = 6800.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


def workload_rho(n, seed=5):
    from paper_2604_13407_gb300 import inputs as I
    return I.spinodal(n, n, 0.5 * (RHO_L + RHO_G), 0.01, seed)


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.device_id = device_id
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.device_id, "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# -------------------------------------------------------------- GPU legs --

def make_sim(n, precision, scheme=1, kernel=0, per_node_ref=1, rounding=1):
    import torch
    from paper_2604_13407_gb300 import lbm
    # FP16 deviations stay below 2^-2 (largest FP16 value 65504 = 2^16 - 2^5); the 2^k
    # scale moves the small ones out of the FP16 subnormal range.
    scale = 18 if precision == lbm.F16DEV else 0
    p = lbm.default_params(nx=n, ny=n, periodic_x=1, periodic_y=1, precision=precision, scheme=scheme,
                           kernel=kernel, per_node_ref=per_node_ref, T=T_07, rho_l=RHO_L, rho_g=RHO_G,
                           rho_s=RHO_G, rho_ref=0.5 * (RHO_L + RHO_G), storage_scale_log2=scale,
                           storage_rounding=rounding, tau_l=TAU, tau_g=TAU)
    return lbm.Simulation(p, stream=torch.cuda.current_stream())


def timed_steps(sim, steps, warmup, dist_on):
    import torch
    sim.step(warmup)
    torch.cuda.synchronize()
    if dist_on:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    sim.step(steps)
    e1.record()
    torch.cuda.synchronize()
    if dist_on:
        torch.distributed.barrier()
    t = e0.elapsed_time(e1) / 1e3
    if dist_on:
        t = max_over_ranks(t)
    return t


def max_over_ranks(t):
    """The largest of the ranks' times (the job ends when the slowest rank ends)."""
    import torch
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([t], device=dev, dtype=torch.float64)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def job_updates(n, steps, world):
    """Lattice updates of the whole job: every rank advances its own n x n replica (weak scaling)."""
    return float(n) * n * steps * world


def e2e_glups(n, precision, steps, rho_host, per_node_ref=1, repeats=3):
    """Same metric through the public API with host buffers: H2D of the initial density
    (pinned), `steps` steps, D2H of rho, ux, uy into pinned host buffers; all inside the
    timed region.  The host copies share the host's memory with whatever else runs on it, so
    the run is repeated and the median reported (with every run's figure)."""
    import torch
    from paper_2604_13407_gb300 import lbm
    sim = make_sim(n, precision, per_node_ref=per_node_ref)
    pinned = torch.from_numpy(rho_host.reshape(-1)).pin_memory()
    out = [torch.empty(n * n, dtype=torch.float64).pin_memory() for _ in range(3)]
    h = pinned.numpy()
    sim.init_fields(h)
    sim.step(2)
    sim.moments(out=out)
    torch.cuda.synchronize()
    runs = []
    for _ in range(repeats):
        gc.collect()  # the earlier legs leave large host arrays behind: no collection inside the timed region
        t0 = time.perf_counter()
        sim.init_fields(h)
        sim.step(steps)
        sim.moments(out=out)  # D2H of rho, ux, uy into pinned host memory (synchronises)
        torch.cuda.synchronize()
        runs.append(n * n * steps / (time.perf_counter() - t0) / 1e9)
    sim.close()
    del out
    return statistics.median(runs), 8 * n * n / steps, 3 * 8 * n * n / steps, runs


def adjoint_cost(precision, nsteps, checkpoint_every=200, nx=256, ny=1024, radius=20.0):
    """Adjoint workload: nx x ny channel (default 256 x 1024; walls at x = -1/2 and nx - 1/2,
    periodic in y), droplet of the given radius (default 20) at a seed-4 jittered centre near
    (nx/2, 0.88 ny), buoyant gravity g = (0, -2e-6), improved scheme.  Times nsteps forward steps and lbm_adjoint_step over
    the same nsteps (forward sweep, segment recompute and transposed steps; objective: the
    y force on the walls; buffers already allocated by a first call) with CUDA events;
    returns the per-step times and their ratio.  FP16 storage: per-node reference density,
    stochastic rounding (the states of the backward sweep are stored in FP16 too)."""
    import torch
    from paper_2604_13407_gb300 import inputs as I
    from paper_2604_13407_gb300 import lbm
    cx, cy = I.jittered_centre(4, nx / 2.0, ny * 900.0 / 1024.0)
    rho = I.droplet(nx, ny, RHO_L, RHO_G, radius, cx, cy, periodic_x=False, periodic_y=True)

    def sim():
        p = lbm.default_params(nx=nx, ny=ny, periodic_x=0, periodic_y=1, precision=precision, scheme=1,
                               force_mode=lbm.FORCE_BUOYANT, Fx=0.0, Fy=-2e-6, T=T_07, rho_l=RHO_L,
                               rho_g=RHO_G, rho_s=RHO_G, tau_l=0.8, tau_g=0.8, per_node_ref=1,
                               storage_scale_log2=18 if precision == lbm.F16DEV else 0)
        s = lbm.Simulation(p, stream=torch.cuda.current_stream())
        s.init_fields(rho)
        return s

    out = {}
    for name in ("forward", "adjoint"):
        s = sim()
        if name == "forward":
            s.step(3)
        else:
            s.adjoint(nsteps, checkpoint_every, lbm.OBJ_WALL_FORCE_Y)  # allocates the checkpoint buffers
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if name == "forward":
            s.step(nsteps)
        else:
            s.adjoint(nsteps, checkpoint_every, lbm.OBJ_WALL_FORCE_Y)
        e1.record()
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / nsteps
        s.close()
    # lbm_adjoint_step advances the state like lbm_step; what it adds is the backward part
    back = out["adjoint"] - out["forward"]
    return {"forward_ms_per_step": out["forward"], "adjoint_ms_per_step": out["adjoint"],
            "ratio": out["adjoint"] / out["forward"], "backward_ms_per_step": back,
            "backward_ratio": back / out["forward"], "steps": nsteps, "checkpoint_every": checkpoint_every,
            "lattice": "%dx%d" % (nx, ny)}


def geometry_cases():
    """Synthetic lattices shaped like the named two-phase configurations, same EOS as the
    headline workload (Carnahan-Starling at 0.7 T_c, eps 1.895), improved scheme:
      oblique_channel_512: 512 x 512 periodic, 45-degree channel between two-node solid bands
        where (x - y) mod 512 < 2, liquid slab across half the width, tau_l = 1.0, tau_g = 0.55,
        force 4e-9 along the bands;
      annulus_1024: 1024 x 1024, solid where r < 128 (at rest) or r > 480 (moving tangentially
        at 0.01), interpolated links, liquid annulus 200 < r < 320, tau 0.8;
      falling_droplet_512x4096: walls at x = -1/2 and 511.5, periodic y, radius-40 droplet at a
        seed-4 jittered centre near (256, 3500), buoyant gravity (rho - rho_g) g, |g| = 2e-6, tau 0.8.
    Yields (name, params overrides, rho, solid, wall_u, q)."""
    from paper_2604_13407_gb300 import inputs as I
    n = 512
    solid = I.oblique_band_walls(n)
    rho = np.where(solid == 1, RHO_G, I.oblique_slab(n, RHO_L, RHO_G, n // 2))
    f = 4e-9 / math.sqrt(2.0)
    yield ("oblique_channel_512", dict(nx=n, ny=n, periodic_x=1, periodic_y=1, Fx=f, Fy=f, tau_l=1.0, tau_g=0.55),
           rho, solid, None, None)
    n = 1024
    solid, wall_u, q = I.annulus(n, n, 128.0, 480.0, u_wall_out=0.01)
    c0 = (n - 1) / 2.0
    r = np.hypot(np.arange(n)[None, :] - c0, np.arange(n)[:, None] - c0)
    ring = RHO_G + 0.5 * (RHO_L - RHO_G) * (np.tanh(2 * (r - 200.0) / 4.0) - np.tanh(2 * (r - 320.0) / 4.0))
    yield ("annulus_1024", dict(nx=n, ny=n, periodic_x=1, periodic_y=1, tau_l=0.8, tau_g=0.8),
           np.where(solid == 1, RHO_G, ring), solid, wall_u, q)
    nx, ny = 512, 4096
    cx, cy = I.jittered_centre(4, 256.0, 3500.0)
    yield ("falling_droplet_512x4096", dict(nx=nx, ny=ny, periodic_x=0, periodic_y=1, force_mode=1, Fy=-2e-6,
                                            tau_l=0.8, tau_g=0.8),
           I.droplet(nx, ny, RHO_L, RHO_G, 40.0, cx, cy, periodic_x=False, periodic_y=True), None, None, None)


def geometry_throughput(hbm, steps=2000, warmup=20, only=None, kernel=0, precs=("f32", "f16dev")):
    """GLUPS of the step on the geometry_cases lattices (CUDA events on the launching
    stream), with the kernel the automatic choice takes ("kernel" names it) unless `kernel`
    asks for one.  Bytes per update (algorithmic): the population read and write of the
    storage type, plus the node's solid flag where there is a mask; interpolated-link
    distances and wall velocities are read only at wall links.  The two smaller lattices'
    state fits in L2 (and the step is bound by latency, not by HBM), so their fraction of the
    HBM copy bandwidth is reported for comparison only.  `only` restricts the run to one
    case (for profiling)."""
    import torch
    from paper_2604_13407_gb300 import lbm
    out = {}
    for name, over, rho, solid, wall_u, q in geometry_cases():
        if only is not None and name != only:
            continue
        for prec in precs:
            pid = {"f64": lbm.F64, "f32": lbm.F32, "f16dev": lbm.F16DEV, "bf16dev": lbm.BF16DEV}[prec]
            half = prec in ("f16dev", "bf16dev")
            p = lbm.default_params(precision=pid, scheme=1, T=T_07, rho_l=RHO_L, rho_g=RHO_G, rho_s=RHO_G,
                                   rho_ref=0.5 * (RHO_L + RHO_G), per_node_ref=1,
                                   storage_scale_log2=18 if prec == "f16dev" else 0, kernel=kernel, **over)
            s = lbm.Simulation(p, stream=torch.cuda.current_stream())
            if solid is not None:
                s.set_geometry(solid, wall_u, q, None)
            s.init_fields(rho)
            nodes = over["nx"] * over["ny"]
            t = timed_steps(s, steps, warmup, False)
            g = nodes * steps / t / 1e9
            b = BYTES[prec] + (8 if half else 0) + (1 if solid is not None else 0)
            # two population buffers (and two reference planes for per-node 16-bit storage)
            state_mb = (BYTES[prec] + (8 if half else 0)) * nodes / 1e6
            out["%s_%s" % (name, prec)] = {
                "GLUPS": g, "us_per_step": 1e6 * t / steps, "bytes_per_update": b, "achieved_GBs": b * g,
                "frac_of_hbm": b * g / hbm, "state_MB": state_mb, "steps": steps,
                "kernel": "fused" if s.kernel_in_use == lbm.KERNEL_FUSED else "two_pass"}
            s.close()
    return out


# ------------------------------------------------------------ CPU legs ----

ORACLE_SAMPLES = {
    "spinodal1024": "1024x1024 periodic spinodal (the 8192x8192 workload's recipe), 100 steps, FP64 oracle",
    "c1": "4x128 grid-aligned two-phase channel (walls in y, F_x = 1e-7, tau 0.8, improved), 20000 steps, FP64 oracle",
}


def oracle_sample(kind, steps=None):
    """Time the FP64 oracle on one bounded sample in this process; returns a dict."""
    from oracle import oracle as O
    if kind == "spinodal1024":
        n = 1024
        p = O.Params(nx=n, ny=n, periodic_x=True, periodic_y=True, scheme=1, T=T_07, rho_l=RHO_L,
                     rho_g=RHO_G, rho_s=RHO_G, tau_l=TAU, tau_g=TAU)
        rho, steps = workload_rho(n), steps or 100
    else:
        from paper_2604_13407_gb300 import inputs as I
        p = O.Params(nx=4, ny=128, periodic_x=True, periodic_y=False, scheme=1, T=T_07, rho_l=RHO_L,
                     rho_g=RHO_G, rho_s=RHO_G, tau_l=0.8, tau_g=0.8, Fx=1e-7)
        rho, steps = I.tanh_slab(4, 128, RHO_L, RHO_G, 64), steps or 20000
    s = O.OracleSim(p)
    s.init(rho)
    s.step(1)
    t0 = time.perf_counter()
    s.step(steps)
    t = time.perf_counter() - t0
    nodes = p.nx * p.ny
    return {"kind": kind, "glups": nodes * steps / t / 1e9, "seconds": t, "steps": steps, "nodes": nodes,
            "threads": O.threads()}


def oracle_in_process(kind, threads, steps=None):
    """oracle_sample in a fresh interpreter with OMP_NUM_THREADS = threads (the OpenMP thread
    count is fixed when the oracle's runtime starts)."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", kind]
    if steps:
        cmd += ["--steps", str(steps)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_cores():
    try:
        return int(subprocess.run(["nproc"], capture_output=True, text=True).stdout.strip())
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline_runs():
    """The CPU baseline: the oracle single-threaded and on every host core, on the spinodal
    sample and on the 4 x 128 channel."""
    cores = host_cores()
    runs = []
    for kind in ("spinodal1024", "c1"):
        for th in (1, cores):
            r = oracle_in_process(kind, th)
            r["sample"] = ORACLE_SAMPLES[kind]
            runs.append(r)
    return cores, runs


def workload_config(n, precision, node_ref=1):
    storage = precision + (" (per-node reference density)" if precision in ("f16dev", "bf16dev") and node_ref else "")
    if precision in ("f16dev", "bf16dev"):
        storage += ", stochastically rounded"
    return {"workload": "spinodal %dx%d periodic, Carnahan-Starling 0.7Tc, eps 1.895, improved "
                        "scheme, tau %.1f, %s population storage" % (n, n, TAU, storage),
            "nx": n, "ny": n, "storage": precision,
            "l2": "inputs larger than L2 (population buffers %.1f GB each)" % (BYTES[precision] / 2 * n * n / 1e9)}


def run_reference(args):
    """The reference arm: the FP64 oracle (the CPU restatement of the paper's step), on every
    host core; each step is one step of a 512 x 512 sample of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.ref_sample
    from oracle import oracle as O
    p = O.Params(nx=n, ny=n, periodic_x=True, periodic_y=True, scheme=1, T=T_07, rho_l=RHO_L,
                 rho_g=RHO_G, rho_s=RHO_G, tau_l=TAU, tau_g=TAU)
    s = O.OracleSim(p)
    s.init(workload_rho(n))
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    t = time.perf_counter() - t0
    v = n * n * args.steps / t / 1e9
    threads = O.threads()
    cfg = workload_config(args.n, args.precision, args.node_ref)
    cfg["parallelism"] = "single"
    sample = "each step: one oracle step of a %dx%d sample of this workload (seed 5), %d host threads" % (n, n, threads)
    line = {"impl": "reference", "metric": "GLUPS", "value": v, "unit": "GLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--precision", default="f32", choices=["f64", "f32", "f16dev", "bf16dev"])
    ap.add_argument("--node-ref", type=int, default=1,
                    help="FP16/BF16 storage: 1 deviations from w_i rho of the writing node (accurate mode), "
                         "0 from one reference density")
    ap.add_argument("--variants", type=int, default=1, help="also time the other precisions / scheme")
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--ref-sample", type=int, default=512)
    ap.add_argument("--e2e", type=int, default=1)
    ap.add_argument("--adjoint", type=int, default=1, help="also time the adjoint against the forward step")
    ap.add_argument("--geometry-only", default=None,
                    choices=("oblique_channel_512", "annulus_1024", "falling_droplet_512x4096"),
                    help="time only this geometry-shaped lattice at --precision (one JSON line; for profiling)")
    ap.add_argument("--kernel", default="auto", choices=("auto", "two_pass", "fused"),
                    help="step kernel for --geometry-only")
    ap.add_argument("--adjoint-only", type=int, default=0,
                    help="time only the adjoint against the forward step (one JSON line; for profiling)")
    ap.add_argument("--adjoint-lattice", type=int, default=0,
                    help="with --adjoint-only: an N x N lattice (droplet radius 160 N/2048, checkpoint every 50) "
                         "instead of the 256 x 1024 channel")
    ap.add_argument("--oracle-sample", default=None, choices=sorted(ORACLE_SAMPLES),
                    help="(internal) time one CPU-baseline sample of the oracle and print it")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.oracle_sample, args.steps if "--steps" in sys.argv else None)))
        return
    if args.impl == "reference":
        return run_reference(args)
    if args.geometry_only:
        import torch
        torch.cuda.set_device(0)
        k = {"auto": 0, "two_pass": 1, "fused": 2}[args.kernel]
        print(json.dumps({"geometry": geometry_throughput(peaks()[0], args.steps, args.warmup, args.geometry_only, k,
                                                          (args.precision,))}))
        return
    if args.adjoint_only:
        import torch
        from paper_2604_13407_gb300 import lbm
        torch.cuda.set_device(0)
        prec = {"f64": lbm.F64, "f32": lbm.F32, "f16dev": lbm.F16DEV}[args.precision]
        N = args.adjoint_lattice
        cost = (adjoint_cost(prec, args.steps, 50, nx=N, ny=N, radius=160.0 * N / 2048.0) if N
                else adjoint_cost(prec, args.steps))
        print(json.dumps({"adjoint": cost, "precision": args.precision}))
        return

    import torch
    from paper_2604_13407_gb300 import lbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist_on = world > 1
    if dist_on:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    prec_id = {"f64": lbm.F64, "f32": lbm.F32, "f16dev": lbm.F16DEV, "bf16dev": lbm.BF16DEV}
    n = args.n
    rho = workload_rho(n, seed=5 + rank)
    hbm, peak_kind = peaks()
    dev_uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    if not dev_uuid.startswith("GPU-"):
        dev_uuid = "GPU-" + dev_uuid

    sim = make_sim(n, prec_id[args.precision], per_node_ref=args.node_ref)
    sim.init_fields(rho)
    kernels_per_step = 1 if sim.kernel_in_use == lbm.KERNEL_FUSED else 2
    with ClockSampler(dev_uuid) as clk:
        t = timed_steps(sim, args.steps, args.warmup, dist_on)
    clocks = clk.summary()
    d = sim.diagnostics()
    sim.close()
    updates = job_updates(n, args.steps, world)
    value = updates / t / 1e9
    bpu = BYTES[args.precision] + (8 if args.precision in ("f16dev", "bf16dev") and args.node_ref else 0)
    # one kernel launch per step on the fused path: the average launch duration is the timed
    # region divided by the steps (CUDA events on the launching stream)
    t_launch = t / args.steps / kernels_per_step
    achieved = bpu * n * n / (t / args.steps) / 1e9

    variants = {}
    if args.variants and rank == 0 and not dist_on:
        for name, prec, scheme, extra in (
                ("f32_original", "f32", 0, {}),
                ("f16dev_node_ref", "f16dev", 1, {"per_node_ref": 1}),
                ("f16dev_node_ref_nearest", "f16dev", 1, {"per_node_ref": 1, "storage_rounding": 0}),
                ("bf16dev_node_ref", "bf16dev", 1, {"per_node_ref": 1}),
                ("f16dev_global_ref", "f16dev", 1, {}),
                ("f64", "f64", 1, {})):
            if prec == args.precision and scheme == 1 and extra.get("storage_rounding", 1) == 1 and (
                    prec in ("f32", "f64") or extra.get("per_node_ref", 0) == args.node_ref):
                continue
            s2 = make_sim(n, prec_id[prec], scheme=scheme, per_node_ref=extra.get("per_node_ref", 0),
                          rounding=extra.get("storage_rounding", 1))
            s2.init_fields(rho)
            k = max(20, args.steps // (4 if prec == "f64" else 1))
            t2 = timed_steps(s2, k, args.warmup, False)
            b = BYTES[prec] + (8 if extra.get("per_node_ref") else 0)
            g = n * n * k / t2 / 1e9
            variants[name] = {"GLUPS": g, "bytes_per_update": b, "achieved_GBs": b * g, "frac": b * g / hbm,
                              "kernel": "fused" if s2.kernel_in_use == lbm.KERNEL_FUSED else "two_pass"}
            if name == "f16dev_node_ref_nearest":
                variants[name]["note"] = "stored deviations rounded to nearest (storage_rounding = 0)"
            if name == "f16dev_global_ref":
                variants[name]["note"] = ("deviations from one reference density, stochastically rounded: about "
                                          "5e-2 of max |u| on the two-phase channel (16x the per-node mode)")
            if prec == "f64":
                # FP64-ALU bound: ncu shows the FP64 pipe busy and DRAM nearly idle (k_fused_f64 profile)
                variants[name]["bound"] = "fp64 alu"
            s2.close()

    geometry = None
    if args.variants and rank == 0 and not dist_on:
        geometry = geometry_throughput(hbm)

    adjoint = None
    if args.adjoint and rank == 0 and not dist_on:
        adjoint = {"workload": "droplet in a 256x1024 channel (radius 20, buoyant g 2e-6, walls in x, periodic y), "
                               "objective: time-averaged y force on the walls, gradient wrt (Fx, Fy, G, T)",
                   "f32": adjoint_cost(lbm.F32, 2000), "f64": adjoint_cost(lbm.F64, 400),
                   "f16dev": adjoint_cost(lbm.F16DEV, 2000),
                   "f32_2048": adjoint_cost(lbm.F32, 200, 50, nx=2048, ny=2048, radius=160.0),
                   "f16dev_2048": adjoint_cost(lbm.F16DEV, 200, 50, nx=2048, ny=2048, radius=160.0)}

    e2e = None
    if rank == 0 and args.e2e:
        ev, hb, db, eruns = e2e_glups(n, prec_id[args.precision], args.steps, rho, args.node_ref)
        e2e = {"value": ev, "unit": "GLUPS", "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db,
               "runs": eruns, "statistic": "median"}
    cpu = None
    if args.cpu_baseline and rank == 0 and not dist_on:
        cores, runs = cpu_baseline_runs()
        head = [r for r in runs if r["kind"] == "spinodal1024" and r["threads"] == cores][0]
        cpu = {"value": head["glups"], "unit": "GLUPS", "cores": head["threads"], "kind": "oracle",
               "sample": head["sample"] + ", %d threads" % head["threads"], "nproc": cores,
               "runs": [{"sample": r["sample"], "threads": r["threads"], "GLUPS": r["glups"], "MLUPS": 1e3 * r["glups"],
                         "seconds": r["seconds"]} for r in runs]}
    if rank == 0:
        cfg = workload_config(n, args.precision, args.node_ref)
        cfg["parallelism"] = "replicas" if world > 1 else "single"
        line = {
            "metric": "GLUPS", "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision != "f64" else "f64",
            "data": "synthetic", "config": cfg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_kind": peak_kind,
                         "traffic": (TRAFFIC_PER_UPDATE[args.precision] * n * n
                                     if kernels_per_step == 1 and TRAFFIC_PER_UPDATE.get(args.precision)
                                     and (args.precision == "f32" or args.node_ref) else None),
                         "traffic_unit": "DRAM bytes per launch (ncu, scaled to this lattice)",
                         "bytes_per_update": bpu, "launch_ms": 1e3 * t_launch,
                         "kernel": "k_fused2" if kernels_per_step == 1 else "two_pass (step)"},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps * kernels_per_step,
            "clocks": clocks, "variants": variants, "geometry": geometry, "adjoint": adjoint,
            "mass": d[0],
        }
        print(json.dumps(line))
    if dist_on:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
