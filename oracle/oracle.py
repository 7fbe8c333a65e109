"""ctypes binding of the FP64 C oracle (les_oracle.c) -- TEST INFRASTRUCTURE ONLY.

The oracle is compiled with plain gcc (``-O2 -fopenmp -ffp-contract=off``, no
fast-math) into ``oracle/liboracle.so`` next to its source.  It receives a
:class:`paper_2301_04698_gb300.inputs.Case`-like object only through its
attribute values; it imports nothing from the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "les_oracle.c")
_HDR = os.path.join(_HERE, "les_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FIELDS = {
    "u": 0, "v": 1, "w": 2, "p": 3, "theta_l": 4, "q_t": 5,
    "u_n": 6, "v_n": 7, "w_n": 8, "theta_l_half": 9, "q_t_half": 10,
    "u_hat": 11, "v_hat": 12, "w_hat": 13, "rhs": 14, "psi": 15,
    "b": 16, "q_l": 17, "T": 18, "s_rad": 19, "nu": 20,
}
NDIAG = 10
DIAG_NAMES = ("sum_rho_theta", "sum_rho_qt", "sum_rho_u", "sum_rho_v", "sum_rho_w",
              "kinetic_energy", "max_cfl", "max_div", "nonfinite", "sum_rho_ql")

_FLAG_BITS = {"adv": 0, "sgs": 1, "const_nu": 2, "moist": 3, "buoy": 4, "coriolis": 5,
              "sponge": 6, "rad": 7, "subs": 8, "sfc": 9, "fb": 10}


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("walls", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("dt", C.c_double), ("cfl", C.c_double),
        ("K", C.c_int32), ("solver", C.c_int32), ("op", C.c_int32), ("warm", C.c_int32),
        ("tol", C.c_double), ("maxit", C.c_int32), ("omega", C.c_double),
        ("flags", C.c_uint32),
        ("cs", C.c_double), ("pr", C.c_double), ("sc", C.c_double), ("nu_const", C.c_double),
        ("f_cor", C.c_double), ("ug", C.c_double), ("vg", C.c_double),
        ("sponge_frac", C.c_double), ("sponge_rate", C.c_double),
        ("subs_div", C.c_double), ("shf", C.c_double), ("lhf", C.c_double),
        ("rad_f0", C.c_double), ("rad_f1", C.c_double), ("rad_kappa", C.c_double),
        ("theta0", C.c_double), ("p00", C.c_double),
        ("sat_tol", C.c_double), ("sat_maxit", C.c_int32), ("advection", C.c_int32),
    ]


def build_oracle(force: bool = False) -> str:
    """Compile les_oracle.c into liboracle.so (once); return the path."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                   "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build_oracle())
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [C.POINTER(_Params), dp]
        lib.orc_destroy.argtypes = [vp]
        lib.orc_field.restype = dp
        lib.orc_field.argtypes = [vp, C.c_int]
        lib.orc_get_dt.restype = C.c_double
        lib.orc_get_dt.argtypes = [vp]
        lib.orc_set_dt.argtypes = [vp, C.c_double]
        lib.orc_profiles.argtypes = [vp, dp, dp]
        lib.orc_begin_step.restype = C.c_int
        lib.orc_begin_step.argtypes = [vp]
        for fn in ("orc_scalar_stage", "orc_momentum_stage", "orc_poisson_rhs", "orc_correct_stage", "orc_end_step"):
            getattr(lib, fn).argtypes = [vp]
        lib.orc_solve_stage.restype = C.c_int
        lib.orc_solve_stage.argtypes = [vp, ip, dp]
        lib.orc_step.restype = C.c_int
        lib.orc_step.argtypes = [vp, C.c_int32, ip]
        lib.orc_apply_poisson.argtypes = [vp, C.c_int32, dp, dp]
        lib.orc_poisson.restype = C.c_int
        lib.orc_poisson.argtypes = [vp, C.c_int32, C.c_int32, dp, dp, C.c_double, C.c_int32, ip, dp]
        lib.orc_nu_field.argtypes = [vp, dp, dp, dp, dp, dp]
        lib.orc_saturation.argtypes = [vp, C.c_int32, C.c_double, C.c_double, dp, dp]
        lib.orc_theta_l_star.restype = C.c_double
        lib.orc_theta_l_star.argtypes = [vp, C.c_int32, C.c_double, C.c_double]
        lib.orc_qv_star.restype = C.c_double
        lib.orc_qv_star.argtypes = [vp, C.c_int32, C.c_double]
        lib.orc_diagnostics.argtypes = [vp, dp]
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One FP64 oracle simulation of a case (attributes as in inputs.Case)."""

    def __init__(self, case, state: dict | None = None):
        lib = _load()
        self.case = case
        self.shape = (case.nz, case.ny, case.nx)
        flags = 0
        for name in case.physics:
            flags |= 1 << _FLAG_BITS[name]
        p = _Params(
            nx=case.nx, ny=case.ny, nz=case.nz, walls=int(bool(case.walls)),
            dx=case.dx, dy=case.dy, dz=case.dz, dt=case.dt, cfl=case.cfl,
            K=case.K, solver={"cg": 0, "jacobi": 1}[case.solver],
            op={"compact": 0, "wide": 1}[case.op],
            warm={"zero": 0, "prev": 1}.get(case.warm, 0),
            tol=case.tol, maxit=case.maxit, omega=case.omega, flags=flags,
            cs=case.cs, pr=case.pr, sc=case.sc, nu_const=case.nu_const,
            f_cor=case.f_cor, ug=case.ug, vg=case.vg,
            sponge_frac=case.sponge_frac, sponge_rate=case.sponge_rate,
            subs_div=case.subs_div, shf=case.shf, lhf=case.lhf,
            rad_f0=case.rad_f0, rad_f1=case.rad_f1, rad_kappa=case.rad_kappa,
            theta0=case.theta0, p00=case.p00,
            sat_tol=1e-10,
            sat_maxit=case.sat_maxit,
            advection={"quick": 0, "weno3": 1}[getattr(case, "advection", "quick")])
        self._params = p
        rho = case.rho0_profile() if hasattr(case, "rho0_profile") else None
        self._rho = _c64(rho) if rho is not None else None
        self._h = lib.orc_create(C.byref(p), _dptr(self._rho) if self._rho is not None else None)
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self._lib = lib
        if state is not None:
            self.set_state(state)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    # -- fields -------------------------------------------------------------
    def view(self, name: str) -> np.ndarray:
        ptr = self._lib.orc_field(self._h, FIELDS[name])
        n = self.shape[0] * self.shape[1] * self.shape[2]
        return np.ctypeslib.as_array(ptr, shape=(n,)).reshape(self.shape)

    def get(self, name: str) -> np.ndarray:
        return self.view(name).copy()

    def set(self, name: str, value) -> None:
        self.view(name)[...] = _c64(value).reshape(self.shape)

    def set_state(self, state: dict) -> None:
        for k in ("u", "v", "w", "p", "theta_l", "q_t"):
            if k in state:
                self.set(k, state[k])

    @property
    def dt(self) -> float:
        return self._lib.orc_get_dt(self._h)

    @dt.setter
    def dt(self, v: float) -> None:
        self._lib.orc_set_dt(self._h, float(v))

    def profiles(self):
        rho = np.zeros(self.shape[0])
        p0 = np.zeros(self.shape[0])
        self._lib.orc_profiles(self._h, _dptr(rho), _dptr(p0))
        return rho, p0

    # -- stages -------------------------------------------------------------
    def begin_step(self) -> None:
        if self._lib.orc_begin_step(self._h):
            raise ValueError("oracle: cannot form a Courant-number time step from a fluid at rest")

    def scalar_stage(self) -> None:
        self._lib.orc_scalar_stage(self._h)

    def momentum_stage(self) -> None:
        self._lib.orc_momentum_stage(self._h)

    def poisson_rhs(self) -> None:
        """the Poisson right side alone, from u^ and psi (the momentum stage
        ends with it)"""
        self._lib.orc_poisson_rhs(self._h)

    def solve_stage(self):
        it = C.c_int32(0)
        res = C.c_double(0.0)
        st = self._lib.orc_solve_stage(self._h, C.byref(it), C.byref(res))
        return st, it.value, res.value

    def correct_stage(self) -> None:
        self._lib.orc_correct_stage(self._h)

    def end_step(self) -> None:
        self._lib.orc_end_step(self._h)

    def step(self, nsteps: int = 1):
        it = C.c_int32(0)
        st = self._lib.orc_step(self._h, int(nsteps), C.byref(it))
        if st == 2:
            raise ValueError("oracle: cannot form a Courant-number time step")
        return st, it.value

    # -- building blocks -----------------------------------------------------
    def apply_poisson(self, x, op: str = "compact") -> np.ndarray:
        x = _c64(x).reshape(-1)
        y = np.zeros_like(x)
        self._lib.orc_apply_poisson(self._h, {"compact": 0, "wide": 1}[op], _dptr(x), _dptr(y))
        return y.reshape(self.shape)

    def poisson(self, b, x0=None, op: str = "compact", solver: str = "cg",
                tol: float = 1e-12, maxit: int = 10000):
        b = _c64(b).reshape(-1)
        x = np.zeros_like(b) if x0 is None else _c64(x0).reshape(-1).copy()
        it = C.c_int32(0)
        res = C.c_double(0.0)
        st = self._lib.orc_poisson(self._h, {"compact": 0, "wide": 1}[op],
                                   {"cg": 0, "jacobi": 1}[solver], _dptr(b), _dptr(x),
                                   float(tol), int(maxit), C.byref(it), C.byref(res))
        return x.reshape(self.shape), st, it.value, res.value

    def nu_field(self, u, v, w, b=None) -> np.ndarray:
        u, v, w = (_c64(a).reshape(-1) for a in (u, v, w))
        bb = _c64(b).reshape(-1) if b is not None else None
        out = np.zeros_like(u)
        self._lib.orc_nu_field(self._h, _dptr(u), _dptr(v), _dptr(w),
                               _dptr(bb) if bb is not None else None, _dptr(out))
        return out.reshape(self.shape)

    def saturation(self, k: int, theta_l: float, q_t: float):
        T = C.c_double(0.0)
        ql = C.c_double(0.0)
        self._lib.orc_saturation(self._h, int(k), float(theta_l), float(q_t),
                                 C.byref(T), C.byref(ql))
        return T.value, ql.value

    def theta_l_star(self, k: int, T: float, q_t: float) -> float:
        return self._lib.orc_theta_l_star(self._h, int(k), float(T), float(q_t))

    def qv_star(self, k: int, T: float) -> float:
        return self._lib.orc_qv_star(self._h, int(k), float(T))

    def diagnostics(self) -> dict:
        out = np.zeros(NDIAG)
        self._lib.orc_diagnostics(self._h, _dptr(out))
        return dict(zip(DIAG_NAMES, out.tolist()))
