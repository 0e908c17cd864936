"""Provenance of tests/golden/table1_aligned_oracle.json: one of its rows (epsilon = 0,
tau = 1.5, original scheme; the cheapest, about 15 s) recomputed here from the oracle with
the same driver (tests/table1.py, oracle backend) must give the stored Err.  The oracle is
deterministic (each thread owns whole rows), so the match is to rounding of the stored
decimal.  Also: LB-ana (Eq. (fde.ali)) from the stored converged densities reproduces the
stored velocities; and the printed Table 1 fixture against the paper's own statements:
the grid-aligned epsilon = 0 row is one value in all four columns (Sec. 3.1), and the
improved scheme's Err is below the original's in every other row."""
import json
import pathlib

import pytest

from tests import table1 as T

GOLD = json.loads((pathlib.Path(__file__).parent / "golden" / "table1_aligned_oracle.json").read_text())["rows"]


def test_stored_oracle_row_is_reproduced():
    row = next(r for r in GOLD if r["epsilon"] == 0.0 and r["tau"] == 1.5 and r["scheme"] == "original")
    # a 181-node column: one thread avoids two OpenMP fork-joins per step on a busy machine
    tpc = pytest.importorskip("threadpoolctl")
    from oracle import oracle as O
    O._load()  # the limit applies to OpenMP runtimes already loaded
    with tpc.threadpool_limits(limits=1, user_api="openmp"):
        err, change, steps, ratio = T.run_aligned(T.OracleBackend(), 0.0, 0.72, 1.5, 0)
    assert abs(err - row["Err"]) <= 1e-12 * row["Err"], (err, row["Err"])
    assert steps == row["steps"]


def test_printed_table_fixture():
    P = T.PAPER
    assert len(set(P["0 aligned"])) == 1
    for key, (o08, o15, i08, i15) in P.items():
        if key != "0 aligned":
            assert i08 < o08 and i15 < o15, key


def _fde_inputs(row):
    """rho, the pairwise force of Eq. (obl.10) (aligned; walls carry psi(rho_s = rho_g)),
    X = F_hat^2 / psi_hat^2, and the stored u of a converged tau = 1.5 row."""
    import numpy as np
    from oracle import analytic as A
    from tests.setups import vdw_params
    rho = np.array(row["profiles"]["rho"])
    u = np.array(row["profiles"]["u"])
    op = vdw_params(row["epsilon"], row["T_r"], nx=1, ny=len(rho))
    psi_hat = np.sqrt(-op.G) * A.psi(rho, 0, op.a, op.b, op.R, op.T, op.K_eos, op.G)
    psi_wall = np.sqrt(-op.G) * A.psi(op.rho_s, 0, op.a, op.b, op.R, op.T, op.K_eos, op.G)
    padded = np.concatenate([[psi_wall], psi_hat, [psi_wall]])
    Fn = psi_hat * (padded[2:] - padded[:-2]) / 2.0
    return rho, Fn, Fn**2 / psi_hat**2, u


@pytest.mark.parametrize("key", [(e, s) for e in (0.0, 1.0, 2.0) for s in ("original", "improved")],
                         ids=lambda k: "eps%g-%s" % k)
def test_lb_ana_reproduces_the_converged_table1_profiles(key):
    """Sec. 3.1, Figs. 3-4 ("LB-ana" agrees with "LB-sim"), on the Table 1 cases themselves:
    Eq. (fde.ali) solved for u from the stored converged density alone (Q_m,6 of
    Eq. (qm6.ali) for the improved scheme; mirror-ghost half-way walls) gives the stored
    velocity to 2e-4 of its maximum (measured 3e-5 to 8e-5) and its Err to 6 %.  The walls
    therefore do not set the small Err values (1e-3) either: those come with the density
    profile and the reading of "Theory"."""
    import numpy as np
    from oracle import analytic as A
    eps, scheme = key
    row = next(r for r in GOLD if r["epsilon"] == eps and r["tau"] == 1.5 and r["scheme"] == scheme)
    rho, Fn, X, u = _fde_inputs(row)
    kq = 3.0 * eps / 8.0 if scheme == "improved" else 0.0
    nu = (1.5 - 0.5) / 3.0
    ua = A.lb_ana_aligned(rho, Fn, X, kq, T.F_DRIVE, nu)
    assert np.abs(ua - u).max() <= 2e-4 * np.abs(u).max()
    th = A.poiseuille_theory(rho, T.F_DRIVE, lambda r: np.full_like(r, nu))
    e_sim, e_ana = A.err_norm(u, th), A.err_norm(ua, th)
    assert abs(e_ana - e_sim) <= 0.06 * e_sim, (e_sim, e_ana)
    assert abs(e_sim - row["Err"]) <= 1e-12 * row["Err"]
