"""The allocation-free FP32 step (lbm_step_noalloc_f32) against the regular entry points.

Callers that cannot call cudaMalloc (stream capture, their own memory pool) use
lbm_step_noalloc_f32 with caller-owned population buffers; its pseudopotential scratch is
a fixed device array inside the library.  Two consecutive calls must give the same
states as lbm_set_state + lbm_step on a context with the two-pass FP32 kernel.
"""
import ctypes

import numpy as np
import pytest

from paper_2604_13407_gb300 import inputs as I
from paper_2604_13407_gb300 import lbm
from tests import gpu_cases as GC
from tests.setups import cs_case, cs_params

pytestmark = pytest.mark.gpu


def _case():
    T, rg, rl = cs_case()
    p = cs_params(nx=96, ny=80, periodic_x=True, periodic_y=False, force_mode=1, Fx=3e-6, Fy=-1e-5, scheme=1)
    return GC.Case("noalloc", p, I.droplet(96, 80, rl, rg, 14, 47.3, 39.6, periodic_x=True, periodic_y=False), 40)


def test_noalloc_step_matches_regular_step_twice():
    import torch
    torch.cuda.set_device(0)
    c = _case()
    ref = GC.run_gpu(c, lbm.F32, lbm.KERNEL_TWO_PASS)      # regular path, 40 steps
    A0 = ref.get_state()
    params = GC.gpu_params(c.params, lbm.F32, lbm.KERNEL_TWO_PASS)
    lib = lbm.load_library()
    ny, nx = c.params.ny, c.params.nx
    pitch = nx + 7                                          # a caller-chosen row pitch
    bufs = [torch.zeros((9, ny, pitch), dtype=torch.float32, device="cuda") for _ in range(2)]
    bufs[0][:, :, :nx] = torch.from_numpy(A0).to(torch.float32)
    stream = torch.cuda.current_stream()
    handle = stream.cuda_stream or 1
    for k in range(2):
        st = lib.lbm_step_noalloc_f32(ctypes.byref(params), ctypes.c_void_p(bufs[k % 2].data_ptr()),
                                      ctypes.c_void_p(bufs[(k + 1) % 2].data_ptr()), pitch, ctypes.c_void_p(handle))
        assert st == 0, lib.lbm_last_error(None)
        torch.cuda.synchronize()
        ref.step(1)
        want = ref.get_state()
        got = bufs[(k + 1) % 2][:, :, :nx].double().cpu().numpy()
        assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max(), k


def test_noalloc_rejects_oversized_and_wrong_precision():
    import torch
    torch.cuda.set_device(0)
    lib = lbm.load_library()
    a = torch.zeros(16, dtype=torch.float32, device="cuda")
    b = torch.zeros(16, dtype=torch.float32, device="cuda")
    big = lbm.default_params(nx=2048, ny=1024, precision=lbm.F32)
    st = lib.lbm_step_noalloc_f32(ctypes.byref(big), ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), 2048, None)
    assert st == 1 and b"LBM_NOALLOC_MAX_NODES" in lib.lbm_last_error(None)
    tall = lbm.default_params(nx=8, ny=70000, precision=lbm.F32)   # 560k nodes, but ny > 65535
    st = lib.lbm_step_noalloc_f32(ctypes.byref(tall), ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), 8, None)
    assert st == 1 and b"65535" in lib.lbm_last_error(None)
    p64 = lbm.default_params(nx=8, ny=8, precision=lbm.F64)
    st = lib.lbm_step_noalloc_f32(ctypes.byref(p64), ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), 8, None)
    assert st == 8
