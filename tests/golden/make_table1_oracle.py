"""Writes table1_aligned_oracle.json: Err of the grid-aligned two-phase Poiseuille flow of
Sec. 3.1 (Table 1) from the FP64 CPU oracle, all twelve aligned cases (epsilon 0, 1, 2;
tau 0.8, 1.5; original and improved Q_m), each run to a relative velocity change below
1e-7 per quarter viscous time by tests/table1.py's converge(), and, for tau = 1.5, the
converged rho and u across the channel.  Only oracle/ computes.

Run from the repository root: `python -m tests.golden.make_table1_oracle` (about ten
minutes on eight cores; one process per case, single-threaded each)."""
import json
import multiprocessing as mp
import os
import pathlib

OUT = pathlib.Path(__file__).parent / "table1_aligned_oracle.json"


def one(args):
    os.environ["OMP_NUM_THREADS"] = "1"
    from tests import table1 as T
    eps, t_r, tau, scheme = args
    row = T.record(T.OracleBackend(), "aligned", eps, t_r, tau, scheme)
    if tau == 1.5:  # the converged profiles, for the LB-ana check of Eq. (fde.ali)
        prof = {}
        T.run_aligned(T.OracleBackend(), eps, t_r, tau, scheme, profiles=prof)
        row["profiles"] = prof
    return row


def main():
    from tests import table1 as T
    jobs = [(eps, t_r, tau, scheme) for eps, t_r in T.CASES for tau in T.TAUS for scheme in (0, 1)]
    os.environ["OMP_NUM_THREADS"] = "1"
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        rows = pool.map(one, jobs)
    OUT.write_text(json.dumps({"source": "FP64 CPU oracle, tests/golden/make_table1_oracle.py",
                               "rows": rows}, indent=1) + "\n")
    for r in rows:
        print(r)


if __name__ == "__main__":
    main()
