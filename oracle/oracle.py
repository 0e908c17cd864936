"""ctypes wrapper around the FP64 C oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU-baseline leg of
bench.py.  The CUDA library and its binding never import this module.

Arrays are numpy float64 in row-major [ny][nx] order (x fastest); population states
are [9][ny][nx] with the D2Q9 numbering e_0 = (0,0), e_1..e_4 = (1,0),(0,1),(-1,0),
(0,-1), e_5..e_8 = (1,1),(-1,1),(-1,-1),(1,-1).
"""
import ctypes
import dataclasses

import numpy as np

from .build import build_oracle

_lib = None


class OrParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("scheme", ctypes.c_int32), ("q2_original", ctypes.c_int32),
        ("eos", ctypes.c_int32), ("force_mode", ctypes.c_int32),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
        ("T", ctypes.c_double), ("K_eos", ctypes.c_double),
        ("G", ctypes.c_double), ("k1", ctypes.c_double), ("k2", ctypes.c_double),
        ("tau_l", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("Lambda", ctypes.c_double),
        ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
        ("rho_s", ctypes.c_double),
    ]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        P = ctypes.POINTER
        d = ctypes.c_double
        dp = P(d)
        lib.or_create.restype = ctypes.c_void_p
        lib.or_create.argtypes = [P(OrParams)]
        lib.or_destroy.argtypes = [ctypes.c_void_p]
        lib.or_set_geometry.argtypes = [ctypes.c_void_p, P(ctypes.c_uint8), dp, dp, dp]
        lib.or_set_wall_density.argtypes = [ctypes.c_void_p, dp]
        lib.or_init.argtypes = [ctypes.c_void_p, dp, dp, dp]
        lib.or_set_state.argtypes = [ctypes.c_void_p, dp]
        lib.or_get_state.argtypes = [ctypes.c_void_p, dp]
        lib.or_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        lib.or_step_count.restype = ctypes.c_int64
        lib.or_step_count.argtypes = [ctypes.c_void_p]
        lib.or_threads.restype = ctypes.c_int
        lib.or_threads.argtypes = []
        lib.or_fields.argtypes = [ctypes.c_void_p] + [dp] * 8
        lib.or_diagnostics.argtypes = [ctypes.c_void_p, dp]
        lib.or_p_eos.restype = d
        lib.or_p_eos.argtypes = [P(OrParams), d]
        lib.or_psi.restype = d
        lib.or_psi.argtypes = [P(OrParams), d]
        lib.or_collide_node.argtypes = [P(OrParams), dp, d, d, d, d, d, dp, dp, dp, dp, dp, dp]
        ip = P(ctypes.c_int)
        lib.or_tables.argtypes = [dp, dp, ip, ip, ip]
        _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


@dataclasses.dataclass
class Params:
    """Problem parameters in the paper's notation (Secs. 2-3)."""
    nx: int = 4
    ny: int = 128
    periodic_x: bool = True
    periodic_y: bool = False
    scheme: int = 1          # 0 original, 1 improved
    q2_original: bool = False
    eos: int = 1             # 0 van der Waals, 1 Carnahan-Starling
    force_mode: int = 0      # 0 constant, 1 (rho - rho_g) g, 2 field
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    T: float = 0.7 * 0.3773 / 4.0
    K_eos: float = 1.0
    G: float = -1.0
    k1: float = -1.895 / 16.0
    k2: float = -1.895 / 16.0
    tau_l: float = 0.8
    tau_g: float = 0.8
    rho_l: float = 0.35814
    rho_g: float = 0.009292
    Lambda: float = 1.0 / 12.0
    Fx: float = 0.0
    Fy: float = 0.0
    rho_s: float = 0.009292

    @property
    def epsilon(self):
        return -8.0 * (self.k1 + self.k2)

    def c_struct(self):
        c = OrParams()
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            setattr(c, f.name, int(v) if isinstance(v, bool) else v)
        return c


def threads() -> int:
    """Threads of the oracle's parallel row loops (OMP_NUM_THREADS at first use)."""
    return int(_load().or_threads())


def p_eos(params: Params, rho: float) -> float:
    c = params.c_struct()
    return _load().or_p_eos(ctypes.byref(c), float(rho))


def psi(params: Params, rho: float) -> float:
    c = params.c_struct()
    return _load().or_psi(ctypes.byref(c), float(rho))


def tables():
    """The oracle's M (9x9), weights, velocities and opposite-direction table."""
    M = np.zeros((9, 9))
    w = np.zeros(9)
    ex = np.zeros(9, dtype=np.intc)
    ey = np.zeros(9, dtype=np.intc)
    opp = np.zeros(9, dtype=np.intc)
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    _load().or_tables(_dp(M), _dp(w), ip(ex), ip(ey), ip(opp))
    return M, w, ex.astype(int), ey.astype(int), opp.astype(int)


def steady_state(sim, warm, rounds=3, settle=20000):
    """Run `warm` steps, then remove the undamped period-2 mode and converge.

    The scheme keeps the staggered momentum sum_x (-1)^(x+y+t) j (both j components)
    exactly: streaming flips the sublattice of every population that carries momentum
    in that direction and the collision adds only the force to j.  A start-up transient
    therefore leaves a period-2 oscillation that never decays.  The average of two
    consecutive states carries that mode only at second order, so restarting from the
    average a few times converges to the time-independent state the paper's steady
    analysis (Sec. 2.1) assumes."""
    sim.step(warm)
    for _ in range(rounds):
        a0 = sim.get_state()
        sim.step(1)
        a1 = sim.get_state()
        sim.set_state(0.5 * (a0 + a1))
        sim.step(settle)
    return sim


def collide_node(params: Params, f, psi_x, S, Fext=(0.0, 0.0)):
    """One-node collision; returns dict(fbar, u, m, meq, Fm, Q)."""
    lib = _load()
    c = params.c_struct()
    f = _f64(f, 9)
    out = {k: np.zeros(9) for k in ("fbar", "m", "meq", "Fm", "Q")}
    out["u"] = np.zeros(2)
    lib.or_collide_node(ctypes.byref(c), _dp(f), float(psi_x), float(S[0]), float(S[1]),
                        float(Fext[0]), float(Fext[1]), _dp(out["fbar"]), _dp(out["u"]),
                        _dp(out["m"]), _dp(out["meq"]), _dp(out["Fm"]), _dp(out["Q"]))
    return out


class OracleSim:
    """FP64 oracle simulation on the CPU."""

    def __init__(self, params: Params, solid=None, wall_u=None, q=None, fext=None, wall_rho=None):
        self.params = params
        self._c = params.c_struct()
        self.n = params.nx * params.ny
        lib = _load()
        self._h = lib.or_create(ctypes.byref(self._c))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self.set_geometry(solid, wall_u, q, fext)
        self.set_wall_density(wall_rho)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().or_destroy(h)
            self._h = None

    def set_geometry(self, solid=None, wall_u=None, q=None, fext=None):
        n = self.n
        self._solid = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        self._wall_u = _f64(wall_u, 2 * n)
        self._q = _f64(q, 8 * n)
        self._fext = _f64(fext, 2 * n)
        sp = None if self._solid is None else self._solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        _load().or_set_geometry(self._h, sp, _dp(self._wall_u), _dp(self._q), _dp(self._fext))

    def set_wall_density(self, wall_rho=None):
        """Virtual density of every solid node ([ny, nx]; read at solid nodes only), or None
        for rho_s at every wall."""
        self._wall_rho = _f64(wall_rho, self.n)
        _load().or_set_wall_density(self._h, _dp(self._wall_rho))

    def init(self, rho, ux=None, uy=None):
        n = self.n
        r = _f64(rho, n)
        ux = _f64(ux, n)
        uy = _f64(uy, n)
        _load().or_init(self._h, _dp(r), _dp(ux), _dp(uy))

    def set_state(self, A):
        A = _f64(A, 9 * self.n)
        _load().or_set_state(self._h, _dp(A))

    def get_state(self):
        A = np.zeros((9, self.params.ny, self.params.nx))
        _load().or_get_state(self._h, _dp(A))
        return A

    def step(self, nsteps=1):
        _load().or_step(self._h, int(nsteps))

    @property
    def step_count(self):
        return _load().or_step_count(self._h)

    def fields(self):
        """dict of rho, ux, uy, Fintx, Finty, psi ([ny][nx]) and Q, f ([9][ny][nx])."""
        ny, nx = self.params.ny, self.params.nx
        out = {k: np.zeros((ny, nx)) for k in ("rho", "ux", "uy", "Fintx", "Finty", "psi")}
        out["Q"] = np.zeros((9, ny, nx))
        out["f"] = np.zeros((9, ny, nx))
        _load().or_fields(self._h, _dp(out["rho"]), _dp(out["ux"]), _dp(out["uy"]),
                          _dp(out["Fintx"]), _dp(out["Finty"]), _dp(out["psi"]),
                          _dp(out["Q"]), _dp(out["f"]))
        return out

    def moments(self):
        f = self.fields()
        return f["rho"], f["ux"], f["uy"]

    def diagnostics(self):
        """[mass, jx, jy, Fx, Fy, wall_x, wall_y, Uc_num, Uc_den, max|u|]"""
        out = np.zeros(10)
        _load().or_diagnostics(self._h, _dp(out))
        return out
