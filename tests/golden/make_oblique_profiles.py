"""Writes oblique_profiles.json: steady 45-degree density profiles rho(alpha) of the
van der Waals set-up of Sec. 3.1 at (epsilon, T_r) = (0, 0.72), (1, 0.65), (2, 0.54), from
the FP64 CPU oracle only.  Each is a periodic 128 x 128 lattice holding a liquid slab 64
alpha-indices wide (alpha = x - y), improved scheme, tau = 1.5, no force, 20000 steps
(mechanical equilibrium of the flat interfaces; max |u| below 2e-4).  The epsilon = 0 slab
starts from densities near its own coexistence (7.29, 0.129) instead of the Maxwell ones,
which lie far from it and throw the run into a violent transient.

Run from the repository root: `python -m tests.golden.make_oblique_profiles` (about two
minutes; one process per case)."""
import json
import multiprocessing as mp
import os
import pathlib

OUT = pathlib.Path(__file__).parent / "oblique_profiles.json"
N, STEPS = 128, 20000
CASES = ((0.0, 0.72, (7.29, 0.129)), (1.0, 0.65, None), (2.0, 0.54, None))


def one(case):
    os.environ["OMP_NUM_THREADS"] = "2"
    import numpy as np
    from oracle import oracle as O
    from paper_2604_13407_gb300 import inputs as I
    from tests.setups import vdw_case, vdw_params
    eps, t_r, start = case
    T, rg, rl = vdw_case(t_r)
    rl0, rg0 = start if start is not None else (rl, rg)
    p = vdw_params(eps, t_r, nx=N, ny=N, periodic_x=True, periodic_y=True, scheme=1, tau_l=1.5, tau_g=1.5)
    s = O.OracleSim(p)
    s.init(I.oblique_slab(N, rl0, rg0, N // 2))
    s.step(STEPS)
    f = s.fields()
    umax = float(np.hypot(f["ux"], f["uy"]).max())
    return {"epsilon": eps, "T_r": t_r, "rho_alpha": [float(v) for v in f["rho"][0, :]], "max_u": umax}


def main():
    with mp.get_context("spawn").Pool(len(CASES)) as pool:
        rows = pool.map(one, CASES)
    OUT.write_text(json.dumps({"source": "FP64 CPU oracle, tests/golden/make_oblique_profiles.py",
                               "n": N, "steps": STEPS, "rows": rows}, indent=1) + "\n")
    for r in rows:
        print(r["epsilon"], r["max_u"], max(r["rho_alpha"]) / min(r["rho_alpha"]))


if __name__ == "__main__":
    main()
