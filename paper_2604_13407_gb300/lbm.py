"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the lattice Boltzmann update runs in liblbm.so; this module only turns
numpy arrays and torch CUDA tensors into the pointers the ABI takes.  Loading fails
with an exception when the library cannot be built or loaded: there is no fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

F64, F32, F16DEV, BF16DEV = 0, 1, 2, 3
ORIGINAL, IMPROVED = 0, 1
EOS_VDW, EOS_CS = 0, 1
FORCE_CONST, FORCE_BUOYANT, FORCE_FIELD = 0, 1, 2
KERNEL_AUTO, KERNEL_TWO_PASS, KERNEL_FUSED = 0, 1, 2
PARAM_FX, PARAM_FY, PARAM_G, PARAM_T = 0, 1, 2, 3
OBJ_WALL_FORCE_Y, OBJ_MEAN_JX = 0, 1
NDIAG = 10

STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_ESTATE",
          5: "LBM_ENAN", 6: "LBM_EBOUNDS", 7: "LBM_ETIMEOUT", 8: "LBM_ENOTSUP"}


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("scheme", ctypes.c_int32),
        ("q2_original", ctypes.c_int32), ("eos", ctypes.c_int32),
        ("force_mode", ctypes.c_int32), ("kernel", ctypes.c_int32),
        ("per_node_ref", ctypes.c_int32), ("storage_scale_log2", ctypes.c_int32),
        ("storage_rounding", ctypes.c_int32), ("diag_every", ctypes.c_int32),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
        ("T", ctypes.c_double), ("K_eos", ctypes.c_double),
        ("G", ctypes.c_double), ("k1", ctypes.c_double), ("k2", ctypes.c_double),
        ("tau_l", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("Lambda", ctypes.c_double), ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
        ("rho_s", ctypes.c_double), ("rho_ref", ctypes.c_double), ("rho_max", ctypes.c_double),
    ]


_lib = None
_P = ctypes.POINTER
_dp = _P(ctypes.c_double)
_vp = ctypes.c_void_p


def load_library(path=None):
    """Build (if needed) and load liblbm.so; raises when that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("LBM_LIBRARY") or _build.build()
    lib = ctypes.CDLL(path)
    st = ctypes.c_int
    sig = {
        "lbm_params_default": (st, [_P(LbmParams)]),
        "lbm_create": (st, [_P(LbmParams), _vp, _P(_vp)]),
        "lbm_destroy": (st, [_vp]),
        "lbm_set_geometry": (st, [_vp, _vp, _vp, _vp, _vp]),
        "lbm_set_wall_density": (st, [_vp, _vp]),
        "lbm_init_fields": (st, [_vp, _vp, _vp, _vp, ctypes.c_int]),
        "lbm_step": (st, [_vp, ctypes.c_int64]),
        "lbm_get_moments": (st, [_vp, _vp, _vp, _vp, ctypes.c_int]),
        "lbm_get_diagnostics": (st, [_vp, _dp]),
        "lbm_get_state": (st, [_vp, _vp, ctypes.c_int]),
        "lbm_set_state": (st, [_vp, _vp, ctypes.c_int]),
        "lbm_save_state": (st, [_vp, _vp, _P(ctypes.c_size_t)]),
        "lbm_load_state": (st, [_vp, _vp, ctypes.c_size_t]),
        "lbm_set_param": (st, [_vp, ctypes.c_int32, ctypes.c_double]),
        "lbm_adjoint_step": (st, [_vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _dp, _dp, _vp]),
        "lbm_sync": (st, [_vp]),
        "lbm_step_count": (ctypes.c_int64, [_vp]),
        "lbm_kernel_in_use": (ctypes.c_int32, [_vp]),
        "lbm_last_error": (ctypes.c_char_p, [_vp]),
        "lbm_step_noalloc_f32": (st, [_P(LbmParams), _vp, _vp, ctypes.c_int64, _vp]),
        "lbm_lb_ana": (st, [_P(LbmParams), ctypes.c_int32, ctypes.c_int32, _dp, _dp, ctypes.c_double, _dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_params(**overrides):
    """lbm_params filled by lbm_params_default, then overridden by keyword."""
    lib = load_library()
    p = LbmParams()
    lib.lbm_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, int(v) if isinstance(v, bool) else v)
    return p


def lb_ana(params, rho, F_drive, oblique=False, f_int=None):
    """lbm_lb_ana: the steady velocity profile the step predicts for the density profile
    rho across a two-phase channel (Eq. (fde.ali), or Eq. (fde.obl) with oblique=True).
    Host arrays; no device is used."""
    lib = load_library()
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    u = np.empty_like(rho)
    fp = None
    if f_int is not None:
        f_int = np.ascontiguousarray(f_int, dtype=np.float64)
        if f_int.shape != rho.shape:
            raise ValueError("f_int must have the shape of rho")
        fp = f_int.ctypes.data_as(_dp)
    st = lib.lbm_lb_ana(ctypes.byref(params), int(bool(oblique)), len(rho), rho.ctypes.data_as(_dp), fp,
                        float(F_drive), u.ctypes.data_as(_dp))
    if st != 0:
        raise LbmError(st, lib.lbm_last_error(None).decode())
    return u


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a, n, dtype=np.float64, keep=None):
    """(pointer, on_device) for a numpy array or torch CUDA tensor of n elements."""
    if a is None:
        return None, None
    if _is_torch_cuda(a):
        import torch
        want = {np.float64: torch.float64, np.uint8: torch.uint8}[dtype]
        if a.dtype != want or not a.is_contiguous() or a.numel() != n:
            raise ValueError("expected a contiguous %s CUDA tensor of %d elements" % (want, n))
        return a.data_ptr(), True
    arr = np.ascontiguousarray(a, dtype=dtype).reshape(-1)
    if arr.size != n:
        raise ValueError("expected %d values, got %d" % (n, arr.size))
    if keep is not None:
        keep.append(arr)
    return arr.ctypes.data, False


class Simulation:
    """One lattice on the current CUDA device (owns an lbm_ctx)."""

    def __init__(self, params=None, stream=None, **overrides):
        """params: LbmParams (see default_params); stream: torch.cuda.Stream, a raw
        cudaStream_t handle, or None for a stream owned by the library.  torch's default
        stream maps to the legacy default stream so torch events order with the steps."""
        self.lib = load_library()
        if params is None:
            params = default_params(**overrides)
        elif overrides:
            for k, v in overrides.items():
                setattr(params, k, v)
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        self.n = self.nx * self.ny
        handle = None
        if stream is not None:
            handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            if handle == 0:
                handle = 1  # the legacy default stream (cudaStreamLegacy), torch's default stream
        h = _vp()
        st = self.lib.lbm_create(ctypes.byref(params), _vp(handle) if handle else None, ctypes.byref(h))
        if st != 0:
            raise LbmError(st, self.lib.lbm_last_error(None).decode())
        self._h = h

    def _check(self, st):
        if st != 0:
            raise LbmError(st, self.lib.lbm_last_error(self._h).decode())

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.lbm_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- set-up
    def set_geometry(self, solid=None, wall_u=None, q=None, force_field=None):
        keep = []
        ps, _ = _ptr(solid, self.n, np.uint8, keep)
        pw, _ = _ptr(wall_u, 2 * self.n, np.float64, keep)
        pq, _ = _ptr(q, 8 * self.n, np.float64, keep)
        pf, _ = _ptr(force_field, 2 * self.n, np.float64, keep)
        self._check(self.lib.lbm_set_geometry(self._h, ps, pw, pq, pf))

    def set_wall_density(self, wall_rho=None):
        """Virtual density of each solid node ([ny, nx], read at solid nodes), or None for
        rho_s at every wall.  A host array: CUDA tensors are copied to the host first."""
        if wall_rho is not None and hasattr(wall_rho, "cpu"):
            wall_rho = wall_rho.detach().cpu().numpy()
        keep = []
        pr, _ = _ptr(wall_rho, self.n, np.float64, keep)
        self._check(self.lib.lbm_set_wall_density(self._h, pr))

    def init_fields(self, rho, ux=None, uy=None):
        keep = []
        pr, dev = _ptr(rho, self.n, keep=keep)
        pu, _ = _ptr(ux, self.n, keep=keep)
        pv, _ = _ptr(uy, self.n, keep=keep)
        self._check(self.lib.lbm_init_fields(self._h, pr, pu, pv, 1 if dev else 0))

    # ---- stepping
    def step(self, nsteps=1):
        self._check(self.lib.lbm_step(self._h, int(nsteps)))

    def sync(self):
        self._check(self.lib.lbm_sync(self._h))

    @property
    def step_count(self):
        return self.lib.lbm_step_count(self._h)

    @property
    def kernel_in_use(self):
        return self.lib.lbm_kernel_in_use(self._h)

    def set_param(self, which, value):
        self._check(self.lib.lbm_set_param(self._h, int(which), float(value)))

    # ---- read-back
    def moments(self, out=None):
        """(rho, ux, uy) as [ny, nx] numpy arrays, or into `out`: three torch CUDA tensors
        (device copies), or three host buffers of nx * ny doubles -- numpy arrays or torch
        CPU tensors, pinned ones for full-speed transfers."""
        if out is not None:
            if all(_is_torch_cuda(a) for a in out):
                r, u, v = out
                self._check(self.lib.lbm_get_moments(self._h, r.data_ptr(), u.data_ptr(), v.data_ptr(), 1))
                return out
            ptrs = []
            for a in out:
                if hasattr(a, "data_ptr"):  # torch CPU tensor
                    if a.dtype != __import__("torch").float64 or not a.is_contiguous() or a.numel() != self.n:
                        raise ValueError("expected a contiguous float64 tensor of %d elements" % self.n)
                    ptrs.append(a.data_ptr())
                else:
                    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != self.n:
                        raise ValueError("expected a contiguous float64 array of %d elements" % self.n)
                    ptrs.append(a.ctypes.data)
            self._check(self.lib.lbm_get_moments(self._h, ptrs[0], ptrs[1], ptrs[2], 0))
            return out
        r = np.zeros((self.ny, self.nx))
        u = np.zeros((self.ny, self.nx))
        v = np.zeros((self.ny, self.nx))
        self._check(self.lib.lbm_get_moments(self._h, r.ctypes.data, u.ctypes.data, v.ctypes.data, 0))
        return r, u, v

    def diagnostics(self):
        out = np.zeros(NDIAG)
        self._check(self.lib.lbm_get_diagnostics(self._h, out.ctypes.data_as(_dp)))
        return out

    def get_state(self, out=None):
        """Decoded populations [9, ny, nx] as FP64 (numpy, or into a torch CUDA tensor)."""
        if out is not None:
            self._check(self.lib.lbm_get_state(self._h, out.data_ptr(), 1))
            return out
        A = np.zeros((9, self.ny, self.nx))
        self._check(self.lib.lbm_get_state(self._h, A.ctypes.data, 0))
        return A

    def set_state(self, A):
        keep = []
        pa, dev = _ptr(A, 9 * self.n, keep=keep)
        self._check(self.lib.lbm_set_state(self._h, pa, 1 if dev else 0))

    def save_state(self):
        nb = ctypes.c_size_t(0)
        self._check(self.lib.lbm_save_state(self._h, None, ctypes.byref(nb)))
        buf = ctypes.create_string_buffer(nb.value)
        self._check(self.lib.lbm_save_state(self._h, buf, ctypes.byref(nb)))
        return buf.raw

    def load_state(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._check(self.lib.lbm_load_state(self._h, buf, len(blob)))

    # ---- adjoint
    def adjoint(self, nsteps, checkpoint_every=200, objective=OBJ_WALL_FORCE_Y, want_lambda0=False,
                want_grad=True):
        """(J, grad[4] = dJ/d(Fx, Fy, G, T) or None, lambda0 or None); advances the state
        nsteps.  want_grad=False and want_lambda0=False run the forward sweep only."""
        J = ctypes.c_double(0)
        g = np.zeros(4) if want_grad else None
        lam = np.zeros((9, self.ny, self.nx)) if want_lambda0 else None
        self._check(self.lib.lbm_adjoint_step(self._h, int(nsteps), int(checkpoint_every), int(objective),
                                              ctypes.byref(J), g.ctypes.data_as(_dp) if g is not None else None,
                                              lam.ctypes.data if lam is not None else None))
        return J.value, g, lam

    def objective(self, nsteps, objective=OBJ_WALL_FORCE_Y):
        """J of nsteps steps from the current state (forward sweep only)."""
        return self.adjoint(nsteps, 1, objective, want_grad=False)[0]


_objective_fn = None


def time_averaged_objective(sim, theta, snapshot, nsteps, checkpoint_every=200, objective=OBJ_WALL_FORCE_Y):
    """J(theta) = (1/nsteps) sum_t J_t of nsteps steps from `snapshot` (lbm_save_state bytes),
    as a torch scalar differentiable in theta = tensor([Fx, Fy, G, T]).  The forward call runs
    lbm_adjoint_step (the gradient comes from the library's transposed-step kernels); the
    backward call scales that gradient by the incoming one."""
    global _objective_fn
    import torch

    if _objective_fn is None:
        class _Objective(torch.autograd.Function):
            @staticmethod
            def forward(ctx, th, sim_, snap, n, k, obj):
                for which, value in enumerate(th.detach().cpu().tolist()):
                    sim_.set_param(which, value)
                sim_.load_state(snap)
                J, g, _ = sim_.adjoint(n, k, obj)
                ctx.save_for_backward(torch.as_tensor(g, dtype=th.dtype, device=th.device))
                return th.new_tensor(J)

            @staticmethod
            def backward(ctx, gJ):
                (g,) = ctx.saved_tensors
                return gJ * g, None, None, None, None, None

        _objective_fn = _Objective
    return _objective_fn.apply(theta, sim, snapshot, int(nsteps), int(checkpoint_every), int(objective))
