"""Host-side checks of the C ABI: the library builds, loads and exports every symbol
include/lbm.h declares; parameter validation rejects bad input before any CUDA call."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2604_13407_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return sorted(set(re.findall(r"^LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_get_moments", "lbm_adjoint_step"):
        assert must in names
    assert len(names) >= 18


def test_library_exports_every_declared_symbol():
    lib = lbm.load_library()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_struct_layout_matches():
    p = lbm.default_params()
    assert p.struct_size == ctypes.sizeof(lbm.LbmParams)
    assert p.nx == 4 and p.ny == 128 and p.precision == lbm.F64
    assert p.k1 == pytest.approx(-1.895 / 16)
    assert p.diag_every == 0 and p.storage_rounding == 1


@pytest.mark.parametrize("field,value", [("nx", 0), ("ny", 65536), ("tau_l", 0.5), ("G", 0.5), ("Lambda", 0.0),
                                         ("precision", 7), ("eos", 3), ("kernel", 9), ("storage_rounding", 2),
                                         ("diag_every", -1)])
def test_create_rejects_invalid_parameters(field, value):
    p = lbm.default_params(**{field: value})
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(p)
    assert e.value.status == 1


@pytest.mark.parametrize("k", [-16, 25])
def test_create_rejects_fp16_scale_outside_the_fp16_range(k):
    """FP16 deviation storage decodes with 2^-k held as an FP16 value: k in [-15, 24]."""
    p = lbm.default_params(precision=lbm.F16DEV, storage_scale_log2=k)
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(p)
    assert e.value.status == 1 and "storage_scale_log2" in str(e.value)


def test_create_rejects_imaginary_pseudopotential():
    # rho_max past the point where p_EOS - rho/3 turns positive (psi^2 < 0)
    p = lbm.default_params(rho_max=0.9)
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(p)
    assert e.value.status == 1 and "psi" in str(e.value)


def test_struct_size_mismatch_rejected():
    p = lbm.default_params()
    p.struct_size = 8
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(p)
    assert e.value.status == 1


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(lbm.default_params())
    assert e.value.status == 3
