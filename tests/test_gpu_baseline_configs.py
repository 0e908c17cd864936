"""The named-configuration driver (tests/baseline_configs.py) end to end at a few hundred
steps: every configuration runs, reports finite figures and agrees with the FP64 oracle over
its prefix (FP64 bit for bit on C2, FP32 within 1e-4 of max |u|).  The full-length runs are
measurements, not tests; this keeps their driver working."""
import math

import pytest

from paper_2604_13407_gb300 import lbm
from tests import baseline_configs as BC

pytestmark = pytest.mark.gpu


def _finite(obj):
    if isinstance(obj, dict):
        return all(_finite(v) for v in obj.values())
    if isinstance(obj, (list, tuple)):
        return all(_finite(v) for v in obj)
    if isinstance(obj, float):
        return math.isfinite(obj)
    return True


def test_c2_short():
    out = BC.c2(lbm, steps=400, prefix=20)
    for scheme, res in out["schemes"].items():
        assert res["f64_vs_oracle_20_steps"] == {"e_u": 0.0, "e_rho": 0.0}, scheme
        assert res["f32_vs_oracle_20_steps"]["e_u"] < 1e-4, scheme
        assert len(res["f32_series"]) == 8 and len(res["f32_tau1_series"]) == 8
        assert _finite(res)


def test_c3_short():
    out = BC.c3(lbm, steps=200, prefix=20, chunk=100, compare_at=100)
    assert out["f32_vs_oracle_20_steps"]["e_u"] < 1e-4
    for name in ("f32", "f16dev_nearest", "f16dev_stochastic", "bf16dev_stochastic", "f32_halfway"):
        assert out[name]["non_finite_at"] is None and len(out[name]["series"]) == 2, name
    assert _finite({k: v for k, v in out.items() if k.endswith("_steps")})


def test_c4_short():
    out = BC.c4(lbm, steps=300, prefix=20, relax=100, samples=3)
    assert out["gas_density"]["with_droplet"] > out["gas_density"]["maxwell"]
    assert out["f32_vs_oracle_20_steps"]["e_u"] < 1e-4
    assert set(out["series"]) == {"%s_%s" % (s, p) for s in ("original", "improved")
                                  for p in ("f32", "f16dev_nearest", "f16dev_stochastic")}
    for rows in out["series"].values():
        assert len(rows) == 3 and all(r["U_c"] is not None and r["R_eq"] > 30 for r in rows)
