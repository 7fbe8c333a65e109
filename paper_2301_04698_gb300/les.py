"""Thin Python binding of libles.so (include/les.h): argument marshalling only.

Every step of the time step runs in the library's CUDA kernels; this module
allocates the device workspace as a torch tensor, passes raw pointers, sizes
and the current torch stream across the C ABI, and converts status codes into
exceptions.  If libles.so is missing it raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libles.so")

# ---- mirrors of include/les.h -----------------------------------------------
LES_OK, LES_ERR_INVALID_ARG, LES_ERR_CUDA, LES_ERR_NOT_CONVERGED = 0, 1, 2, 3
LES_ERR_NONFINITE, LES_ERR_TIMEOUT, LES_ERR_STATE, LES_ERR_NO_MODEL = 4, 5, 6, 7

PHYS_BITS = {"adv": 1 << 0, "sgs": 1 << 1, "const_nu": 1 << 2, "moist": 1 << 3, "buoy": 1 << 4,
             "coriolis": 1 << 5, "sponge": 1 << 6, "rad": 1 << 7, "subs": 1 << 8, "sfc": 1 << 9,
             "fb": 1 << 10}
FIELDS = {"u": 0, "v": 1, "w": 2, "p": 3, "theta_l": 4, "q_t": 5, "u_n": 6, "v_n": 7, "w_n": 8,
          "theta_l_half": 9, "q_t_half": 10, "u_hat": 11, "v_hat": 12, "w_hat": 13, "rhs": 14,
          "psi": 15, "b": 16, "q_l": 17, "T": 18, "s_rad": 19}
STAGES = {"begin": 0, "scalar": 1, "momentum": 2, "solve": 3, "correct": 4, "end": 5}
SOLVERS = {"cg": 0, "jacobi": 1}
OPS = {"compact": 0, "wide": 1}
WARM = {"zero": 0, "prev": 1, "learned": 2}
NDIAG = 10
DIAG_NAMES = ("sum_rho_theta", "sum_rho_qt", "sum_rho_u", "sum_rho_v", "sum_rho_w",
              "kinetic_energy", "max_cfl", "max_div", "nonfinite", "sum_rho_ql")

#: every symbol declared in include/les.h
EXPORTED = ("les_config_default", "les_workspace_bytes", "les_init", "les_destroy", "les_set_stream",
            "les_set_state", "les_get_state", "les_field_offset", "les_step", "les_stage",
            "les_poisson_solve", "les_apply_poisson", "les_diagnostics", "les_get_dt", "les_set_dt",
            "les_last_error", "les_status_string", "les_profile_enable", "les_profile_read",
            "les_profile_reset", "les_launch_count", "les_poisson_solve_static", "les_get_tuning",
            "les_set_tuning", "les_unet_param_count", "les_unet_workspace_bytes", "les_unet_create",
            "les_unet_destroy", "les_unet_set_stream", "les_unet_set_weights", "les_unet_get_weights",
            "les_unet_forward", "les_unet_loss_grad", "les_unet_train_step", "les_unet_last_error",
            "les_set_warm_model", "les_unet_set_output_scale", "les_unet_get_output_scale", "les_unet_set_loss",
            "les_ensemble_step", "les_set_states", "les_dd_workspace_bytes", "les_dd_create", "les_dd_destroy",
            "les_dd_local_shape", "les_dd_poisson_solve", "les_dd_last_error", "les_dd_step_config",
            "les_dd_halo_exchange", "les_dd_stage_solve", "les_prefetch_states", "les_measure_fma")


class LesConfig(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("precision", C.c_int32),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("bc_z", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("dt", C.c_double), ("cfl", C.c_double),
        ("n_subiter", C.c_int32), ("solver", C.c_int32), ("poisson_op", C.c_int32),
        ("warm_start", C.c_int32),
        ("poisson_tol", C.c_double), ("poisson_maxit", C.c_int32), ("physics", C.c_uint32),
        ("jacobi_omega", C.c_double), ("cs", C.c_double), ("pr", C.c_double), ("sc", C.c_double),
        ("const_nu", C.c_double), ("f_cor", C.c_double), ("ug", C.c_double), ("vg", C.c_double),
        ("sponge_frac", C.c_double), ("sponge_rate", C.c_double), ("subs_div", C.c_double),
        ("shf", C.c_double), ("lhf", C.c_double), ("rad_f0", C.c_double), ("rad_f1", C.c_double),
        ("rad_kappa", C.c_double), ("theta0", C.c_double), ("p00", C.c_double),
        ("sat_tol", C.c_double), ("sat_maxit", C.c_int32), ("solver_path", C.c_int32),
        ("advection", C.c_int32), ("precond", C.c_int32), ("reserved", C.c_double * 3),
    ]


class LesStepStats(C.Structure):
    _fields_ = [("steps", C.c_int32), ("solves", C.c_int32), ("iters_total", C.c_int32),
                ("iters_max", C.c_int32), ("not_converged", C.c_int32), ("reserved0", C.c_int32),
                ("res_max", C.c_double), ("dt", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class LesKernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("fields_per_cell", C.c_int32), ("reserved0", C.c_int32),
                ("launches", C.c_int64), ("timed", C.c_int64), ("total_ms", C.c_double),
                ("bytes_per_launch", C.c_double)]


class LesTuning(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("cg_tile_rows", C.c_int32), ("cg_tile_planes", C.c_int32),
                ("cg_max_blocks", C.c_int32), ("barrier_timeout_ms", C.c_double),
                ("fault_missing_arrivals", C.c_int32), ("stencil_path", C.c_int32), ("cg_variant", C.c_int32),
                ("cg_resident", C.c_int32)]


class LesError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libles.so.  Raises if it has not been built -- never falls back."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2301_04698_gb300.build.build() "
                           "(the LES path has no CPU fallback)")
    lib = C.CDLL(path)
    vp, i32, dbl, sz = C.c_void_p, C.c_int32, C.c_double, C.c_size_t
    cfgp = C.POINTER(LesConfig)
    statp = C.POINTER(LesStepStats)
    lib.les_config_default.restype = None
    lib.les_config_default.argtypes = [cfgp, i32, i32, i32]
    lib.les_workspace_bytes.restype = C.c_int
    lib.les_workspace_bytes.argtypes = [cfgp, C.POINTER(sz)]
    lib.les_init.restype = C.c_int
    lib.les_init.argtypes = [cfgp, C.POINTER(dbl), vp, sz, vp, C.POINTER(vp)]
    lib.les_destroy.restype = None
    lib.les_destroy.argtypes = [vp]
    lib.les_set_stream.restype = C.c_int
    lib.les_set_stream.argtypes = [vp, vp]
    lib.les_set_state.restype = C.c_int
    lib.les_set_state.argtypes = [vp, i32, vp, i32]
    lib.les_set_states.restype = C.c_int
    lib.les_set_states.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(vp), i32]
    lib.les_get_state.restype = C.c_int
    lib.les_get_state.argtypes = [vp, i32, vp, i32]
    lib.les_field_offset.restype = C.c_int
    lib.les_field_offset.argtypes = [vp, i32, C.POINTER(sz)]
    lib.les_step.restype = C.c_int
    lib.les_step.argtypes = [vp, i32, statp]
    lib.les_stage.restype = C.c_int
    lib.les_stage.argtypes = [vp, i32, statp]
    lib.les_ensemble_step.restype = C.c_int
    lib.les_ensemble_step.argtypes = [C.POINTER(vp), i32, i32, statp, C.POINTER(i32)]
    lib.les_poisson_solve.restype = C.c_int
    lib.les_poisson_solve.argtypes = [vp, vp, vp, dbl, i32, C.POINTER(i32), C.POINTER(dbl)]
    lib.les_apply_poisson.restype = C.c_int
    lib.les_apply_poisson.argtypes = [vp, i32, vp, vp]
    lib.les_diagnostics.restype = C.c_int
    lib.les_diagnostics.argtypes = [vp, C.POINTER(dbl)]
    lib.les_get_dt.restype = dbl
    lib.les_get_dt.argtypes = [vp]
    lib.les_set_dt.restype = C.c_int
    lib.les_set_dt.argtypes = [vp, dbl]
    lib.les_last_error.restype = C.c_char_p
    lib.les_last_error.argtypes = [vp]
    lib.les_status_string.restype = C.c_char_p
    lib.les_status_string.argtypes = [C.c_int]
    lib.les_profile_enable.restype = C.c_int
    lib.les_profile_enable.argtypes = [vp, i32]
    lib.les_profile_read.restype = C.c_int
    lib.les_profile_read.argtypes = [vp, C.POINTER(LesKernelStat), i32, C.POINTER(i32)]
    lib.les_profile_reset.restype = C.c_int
    lib.les_profile_reset.argtypes = [vp]
    lib.les_launch_count.restype = C.c_int64
    lib.les_launch_count.argtypes = [vp]
    lib.les_get_tuning.restype = C.c_int
    lib.les_get_tuning.argtypes = [vp, C.POINTER(LesTuning)]
    lib.les_set_tuning.restype = C.c_int
    lib.les_set_tuning.argtypes = [vp, C.POINTER(LesTuning)]
    lib.les_unet_param_count.restype = C.c_int64
    lib.les_unet_param_count.argtypes = []
    lib.les_unet_workspace_bytes.restype = C.c_int
    lib.les_unet_workspace_bytes.argtypes = [i32, i32, C.POINTER(sz)]
    lib.les_unet_create.restype = C.c_int
    lib.les_unet_create.argtypes = [i32, i32, vp, sz, vp, C.POINTER(vp)]
    lib.les_unet_destroy.restype = None
    lib.les_unet_destroy.argtypes = [vp]
    lib.les_unet_set_stream.restype = C.c_int
    lib.les_unet_set_stream.argtypes = [vp, vp]
    lib.les_unet_set_weights.restype = C.c_int
    lib.les_unet_set_weights.argtypes = [vp, vp, i32]
    lib.les_unet_get_weights.restype = C.c_int
    lib.les_unet_get_weights.argtypes = [vp, vp, i32]
    lib.les_unet_forward.restype = C.c_int
    lib.les_unet_forward.argtypes = [vp, i32, vp, i32, vp]
    lib.les_unet_loss_grad.restype = C.c_int
    lib.les_unet_loss_grad.argtypes = [vp, i32, vp, vp, i32, C.POINTER(dbl), vp]
    lib.les_unet_train_step.restype = C.c_int
    lib.les_unet_train_step.argtypes = [vp, i32, vp, vp, i32, C.c_float, C.POINTER(dbl)]
    lib.les_unet_last_error.restype = C.c_char_p
    lib.les_unet_last_error.argtypes = [vp]
    lib.les_unet_set_output_scale.restype = C.c_int
    lib.les_unet_set_output_scale.argtypes = [vp, dbl]
    lib.les_unet_get_output_scale.restype = dbl
    lib.les_unet_get_output_scale.argtypes = [vp]
    lib.les_unet_set_loss.restype = C.c_int
    lib.les_unet_set_loss.argtypes = [vp, C.c_int32]
    lib.les_dd_workspace_bytes.restype = C.c_int
    lib.les_dd_workspace_bytes.argtypes = [cfgp, i32, i32, C.POINTER(sz)]
    lib.les_dd_create.restype = C.c_int
    lib.les_dd_create.argtypes = [cfgp, i32, i32, i32, i32, vp, sz, vp, C.POINTER(vp)]
    lib.les_dd_destroy.restype = None
    lib.les_dd_destroy.argtypes = [vp]
    lib.les_dd_local_shape.restype = C.c_int
    lib.les_dd_local_shape.argtypes = [vp] + [C.POINTER(i32)] * 5
    lib.les_dd_poisson_solve.restype = C.c_int
    lib.les_dd_poisson_solve.argtypes = [vp, vp, vp, vp, dbl, i32, C.POINTER(i32), C.POINTER(dbl)]
    lib.les_dd_last_error.restype = C.c_char_p
    lib.les_dd_last_error.argtypes = [vp]
    lib.les_prefetch_states.restype = C.c_int
    lib.les_prefetch_states.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(vp), vp, vp]
    lib.les_dd_step_config.restype = C.c_int
    lib.les_dd_step_config.argtypes = [vp, cfgp]
    lib.les_dd_halo_exchange.restype = C.c_int
    lib.les_dd_halo_exchange.argtypes = [vp, vp, vp, i32, C.POINTER(i32)]
    lib.les_dd_stage_solve.restype = C.c_int
    lib.les_dd_stage_solve.argtypes = [vp, vp, vp, C.POINTER(LesStepStats)]
    lib.les_set_warm_model.restype = C.c_int
    lib.les_set_warm_model.argtypes = [vp, vp]
    lib.les_poisson_solve_static.restype = C.c_int
    lib.les_poisson_solve_static.argtypes = [cfgp, vp, vp, vp, dbl, i32, vp, C.POINTER(i32), C.POINTER(dbl),
                                             C.c_char_p, sz]
    lib.les_measure_fma.restype = C.c_int
    lib.les_measure_fma.argtypes = [vp, i32, i32, C.POINTER(dbl), C.POINTER(dbl)]
    _lib = lib
    return lib


def measure_fma(precision: int = 32, trips: int = 10000, stream=None) -> dict:
    """The device's FMA rate in FP32 or FP64 (les_measure_fma): {"tflops", "ms"}."""
    lib = load_library()
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    rc = lib.les_measure_fma(C.c_void_p(stream.cuda_stream if stream is not None else 0), int(precision), int(trips),
                             C.byref(tf), C.byref(ms))
    if rc != LES_OK:
        raise LesError(rc, f"les_measure_fma: status {rc}")
    return {"tflops": tf.value, "ms": ms.value}


def config_from_case(case) -> LesConfig:
    """les_config for a workload description (attributes as in inputs.Case)."""
    lib = load_library()
    c = LesConfig()
    lib.les_config_default(C.byref(c), case.nx, case.ny, case.nz)
    c.precision = int(case.precision)
    c.bc_z = 1 if case.walls else 0
    c.dx, c.dy, c.dz = float(case.dx), float(case.dy), float(case.dz)
    c.dt, c.cfl = float(case.dt), float(case.cfl)
    c.n_subiter = int(case.K)
    c.solver = SOLVERS[case.solver]
    c.poisson_op = OPS[case.op]
    c.warm_start = WARM[case.warm]
    c.poisson_tol, c.poisson_maxit = float(case.tol), int(case.maxit)
    phys = 0
    for name in case.physics:
        phys |= PHYS_BITS[name]
    c.physics = phys
    c.jacobi_omega = float(case.omega)
    for k in ("cs", "pr", "sc", "f_cor", "ug", "vg", "sponge_frac", "sponge_rate", "subs_div", "shf",
              "lhf", "rad_f0", "rad_f1", "rad_kappa", "theta0", "p00", "sat_tol"):
        setattr(c, k, float(getattr(case, k)))
    c.const_nu = float(case.nu_const)
    c.sat_maxit = int(case.sat_maxit)
    c.solver_path = int(getattr(case, "solver_path", 0))
    c.advection = {"quick": 0, "weno3": 1}[getattr(case, "advection", "quick")]
    c.precond = {"none": 0, "learned": 1}[getattr(case, "precond", "none")]
    return c


def _check(lib, h, rc, what, allow=(LES_OK,)):
    if rc in allow:
        return rc
    msg = lib.les_last_error(h).decode() if h else lib.les_status_string(rc).decode()
    raise LesError(rc, f"{what}: {lib.les_status_string(rc).decode()}: {msg}")


class Simulation:
    """One LES on the current CUDA device, behind the C ABI."""

    def __init__(self, case, device=None, stream=None):
        import torch
        self.torch = torch
        self.lib = lib = load_library()
        self.case = case
        self.cfg = config_from_case(case)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.dtype = torch.float64 if case.precision == 64 else torch.float32
        self.np_dtype = np.float64 if case.precision == 64 else np.float32
        self.shape = (case.nz, case.ny, case.nx)
        self.n = case.nx * case.ny * case.nz
        self.esize = 8 if case.precision == 64 else 4
        nbytes = C.c_size_t(0)
        _check(lib, None, lib.les_workspace_bytes(C.byref(self.cfg), C.byref(nbytes)), "les_workspace_bytes")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        rho = case.rho0_profile() if hasattr(case, "rho0_profile") else None
        self._rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        h = C.c_void_p()
        rc = lib.les_init(C.byref(self.cfg),
                          self._rho.ctypes.data_as(C.POINTER(C.c_double)) if self._rho is not None else None,
                          C.c_void_p(self.workspace.data_ptr()), nbytes, C.c_void_p(self.stream.cuda_stream),
                          C.byref(h))
        _check(lib, None, rc, "les_init")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.les_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- fields ---------------------------------------------------------------
    def view(self, name: str):
        """Zero-copy torch view of a field's current buffer (shape nz, ny, nx)."""
        off = C.c_size_t(0)
        _check(self.lib, self.h, self.lib.les_field_offset(self.h, FIELDS[name], C.byref(off)), "offset")
        raw = self.workspace[off.value: off.value + self.n * self.esize]
        return raw.view(self.dtype).view(self.shape)

    def set(self, name: str, value) -> None:
        t = self.torch
        if isinstance(value, np.ndarray):
            src = t.from_numpy(np.ascontiguousarray(value.reshape(self.shape), dtype=self.np_dtype))
            src = src.to(self.device, non_blocking=False)
        else:
            src = value.reshape(self.shape).to(device=self.device, dtype=self.dtype).contiguous()
        with t.cuda.stream(self.stream):
            rc = self.lib.les_set_state(self.h, FIELDS[name], C.c_void_p(src.data_ptr()), 1)
        _check(self.lib, self.h, rc, f"set {name}")
        self.stream.synchronize()

    def set_state(self, state: dict) -> None:
        for k in ("u", "v", "w", "p", "theta_l", "q_t"):
            if k in state:
                self.set(k, state[k])

    def set_from_host(self, name: str, host) -> None:
        """Host-buffer transfer through the ABI (host pointer, synchronous)."""
        rc = self.lib.les_set_state(self.h, FIELDS[name], C.c_void_p(host.data_ptr()), 0)
        _check(self.lib, self.h, rc, f"set {name} (host)")

    def set_many_from_host(self, hosts: dict) -> None:
        """Host-buffer transfer of several fields through one ABI call (all
        copies enqueued, one synchronisation)."""
        names = list(hosts)
        ids = (C.c_int32 * len(names))(*[FIELDS[k] for k in names])
        ptrs = (C.c_void_p * len(names))(*[C.c_void_p(hosts[k].data_ptr()) for k in names])
        rc = self.lib.les_set_states(self.h, len(names), ids, ptrs, 0)
        _check(self.lib, self.h, rc, "set states (host)")

    def prefetch_from_host(self, hosts: dict, staging, stream) -> None:
        """les_prefetch_states: hosts[name] (pinned torch tensors) into the
        device buffer `staging` (torch tensor of at least len(hosts) fields)
        on `stream` (a torch.cuda.Stream); the next BEGIN takes them."""
        names = list(hosts)
        if staging.numel() * staging.element_size() < len(names) * self.n * self.esize:
            raise ValueError("staging buffer too small")
        ids = (C.c_int32 * len(names))(*[FIELDS[k] for k in names])
        ptrs = (C.c_void_p * len(names))(*[C.c_void_p(hosts[k].data_ptr()) for k in names])
        rc = self.lib.les_prefetch_states(self.h, len(names), ids, ptrs, C.c_void_p(staging.data_ptr()),
                                          C.c_void_p(stream.cuda_stream))
        _check(self.lib, self.h, rc, "prefetch states")

    def get_to_host(self, name: str, host) -> None:
        rc = self.lib.les_get_state(self.h, FIELDS[name], C.c_void_p(host.data_ptr()), 0)
        _check(self.lib, self.h, rc, f"get {name} (host)")

    def get(self, name: str) -> np.ndarray:
        out = np.empty(self.shape, dtype=self.np_dtype)
        rc = self.lib.les_get_state(self.h, FIELDS[name], C.c_void_p(out.ctypes.data), 0)
        _check(self.lib, self.h, rc, f"get {name}")
        return out

    # -- stepping -------------------------------------------------------------
    def step(self, nsteps: int = 1, allow_not_converged: bool = False) -> dict:
        st = LesStepStats()
        allow = (LES_OK, LES_ERR_NOT_CONVERGED) if allow_not_converged else (LES_OK,)
        rc = self.lib.les_step(self.h, int(nsteps), C.byref(st))
        _check(self.lib, self.h, rc, "les_step", allow)
        d = st.as_dict()
        d["status"] = rc
        return d

    def stage(self, name: str, allow_not_converged: bool = False) -> dict:
        st = LesStepStats()
        allow = (LES_OK, LES_ERR_NOT_CONVERGED) if allow_not_converged else (LES_OK,)
        rc = self.lib.les_stage(self.h, STAGES[name], C.byref(st))
        _check(self.lib, self.h, rc, f"les_stage({name})", allow)
        d = st.as_dict()
        d["status"] = rc
        return d

    @property
    def dt(self) -> float:
        return self.lib.les_get_dt(self.h)

    @dt.setter
    def dt(self, v: float) -> None:
        _check(self.lib, self.h, self.lib.les_set_dt(self.h, float(v)), "les_set_dt")

    # -- solver ---------------------------------------------------------------
    def poisson_solve(self, rhs, x, tol: float, maxit: int, allow_not_converged: bool = False):
        it = C.c_int32(0)
        rel = C.c_double(0.0)
        rc = self.lib.les_poisson_solve(self.h, C.c_void_p(rhs.data_ptr()), C.c_void_p(x.data_ptr()),
                                        float(tol), int(maxit), C.byref(it), C.byref(rel))
        allow = (LES_OK, LES_ERR_NOT_CONVERGED) if allow_not_converged else (LES_OK,)
        _check(self.lib, self.h, rc, "les_poisson_solve", allow)
        return rc, it.value, rel.value

    def apply_poisson(self, x, op: str = "compact"):
        y = self.torch.empty_like(x)
        rc = self.lib.les_apply_poisson(self.h, OPS[op], C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()))
        _check(self.lib, self.h, rc, "les_apply_poisson")
        return y

    # -- profiling ------------------------------------------------------------
    def profile(self, enable: bool) -> None:
        _check(self.lib, self.h, self.lib.les_profile_enable(self.h, int(bool(enable))), "profile")

    def profile_reset(self) -> None:
        _check(self.lib, self.h, self.lib.les_profile_reset(self.h), "profile reset")

    def profile_read(self) -> list:
        arr = (LesKernelStat * 32)()
        cnt = C.c_int32(0)
        _check(self.lib, self.h, self.lib.les_profile_read(self.h, arr, 32, C.byref(cnt)), "profile read")
        out = []
        for k in arr[:cnt.value]:
            out.append({"name": k.name.decode(), "fields_per_cell": k.fields_per_cell,
                        "launches": k.launches, "timed": k.timed, "total_ms": k.total_ms,
                        "bytes_per_launch": k.bytes_per_launch})
        return out

    def tuning(self) -> dict:
        t = LesTuning()
        _check(self.lib, self.h, self.lib.les_get_tuning(self.h, C.byref(t)), "get tuning")
        return {k: getattr(t, k) for k, _ in t._fields_ if k not in ("struct_size", "reserved0")}

    def set_tuning(self, **kw) -> None:
        t = LesTuning()
        t.struct_size = C.sizeof(LesTuning)
        cur = self.tuning()
        t.stencil_path = cur["stencil_path"]
        t.cg_variant = cur["cg_variant"]
        t.cg_resident = cur["cg_resident"]
        for k, v in kw.items():
            setattr(t, k, v)
        _check(self.lib, self.h, self.lib.les_set_tuning(self.h, C.byref(t)), "set tuning")

    def launch_count(self) -> int:
        return int(self.lib.les_launch_count(self.h))

    def diagnostics(self) -> dict:
        out = (C.c_double * NDIAG)()
        rc = self.lib.les_diagnostics(self.h, out)
        _check(self.lib, self.h, rc, "les_diagnostics", (LES_OK, LES_ERR_NONFINITE))
        return dict(zip(DIAG_NAMES, list(out)))


class UNet:
    """The learned warm-start network behind the C ABI (les_unet_*)."""

    def __init__(self, n: int, max_batch: int = 1, device=None, stream=None):
        import torch
        self.torch = torch
        self.lib = lib = load_library()
        self.n, self.max_batch = int(n), int(max_batch)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nbytes = C.c_size_t(0)
        rc = lib.les_unet_workspace_bytes(self.n, self.max_batch, C.byref(nbytes))
        _check(lib, None, rc, "les_unet_workspace_bytes")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        rc = lib.les_unet_create(self.n, self.max_batch, C.c_void_p(self.workspace.data_ptr()), nbytes,
                                 C.c_void_p(self.stream.cuda_stream), C.byref(h))
        _check(lib, None, rc, "les_unet_create")
        self.h = h
        self.nparams = int(lib.les_unet_param_count())

    def close(self):
        if getattr(self, "h", None):
            self.lib.les_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc, what):
        if rc != LES_OK:
            raise LesError(rc, f"{what}: {self.lib.les_unet_last_error(self.h).decode()}")

    def set_weights(self, w) -> None:
        t = self.torch
        wt = t.as_tensor(np.asarray(w, dtype=np.float32) if not isinstance(w, t.Tensor) else w,
                         dtype=t.float32).to(self.device).contiguous()
        assert wt.numel() == self.nparams
        self._ck(self.lib.les_unet_set_weights(self.h, C.c_void_p(wt.data_ptr()), 1), "set_weights")
        self.stream.synchronize()

    @property
    def out_scale(self) -> float:
        return float(self.lib.les_unet_get_output_scale(self.h))

    @out_scale.setter
    def out_scale(self, v: float) -> None:
        self._ck(self.lib.les_unet_set_output_scale(self.h, float(v)), "set_output_scale")

    def set_loss(self, kind: str) -> None:
        """Training loss: "mse" or "energy" (energy norm of the error)."""
        self._ck(self.lib.les_unet_set_loss(self.h, {"mse": 0, "energy": 1}[kind]), "set_loss")

    def get_weights(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        self._ck(self.lib.les_unet_get_weights(self.h, C.c_void_p(out.ctypes.data), 0), "get_weights")
        return out

    def forward(self, b):
        """psi_0 for a (batch, n, n, n) or (n, n, n) tensor of right-hand sides."""
        psi = self.torch.empty_like(b)
        batch = b.numel() // self.n ** 3
        prec = 64 if b.dtype == self.torch.float64 else 32
        self._ck(self.lib.les_unet_forward(self.h, prec, C.c_void_p(b.data_ptr()), batch,
                                           C.c_void_p(psi.data_ptr())), "forward")
        return psi

    def loss_grad(self, b, psi):
        grad = self.torch.empty(self.nparams, dtype=self.torch.float32, device=self.device)
        loss = C.c_double(0.0)
        batch = b.numel() // self.n ** 3
        prec = 64 if b.dtype == self.torch.float64 else 32
        self._ck(self.lib.les_unet_loss_grad(self.h, prec, C.c_void_p(b.data_ptr()), C.c_void_p(psi.data_ptr()),
                                             batch, C.byref(loss), C.c_void_p(grad.data_ptr())), "loss_grad")
        return loss.value, grad

    def train_step(self, b, psi, lr: float, want_loss: bool = True):
        loss = C.c_double(0.0)
        batch = b.numel() // self.n ** 3
        prec = 64 if b.dtype == self.torch.float64 else 32
        self._ck(self.lib.les_unet_train_step(self.h, prec, C.c_void_p(b.data_ptr()), C.c_void_p(psi.data_ptr()),
                                              batch, float(lr), C.byref(loss) if want_loss else None),
                 "train_step")
        return loss.value if want_loss else None


def attach_model(sim: "Simulation", model) -> None:
    """Use `model` for LES_WARM_LEARNED solves of `sim` (None detaches)."""
    rc = sim.lib.les_set_warm_model(sim.h, model.h if model is not None else None)
    _check(sim.lib, sim.h, rc, "les_set_warm_model")
    sim._model = model


class Ensemble:
    """Independent members (each its own Simulation and stream) stepped
    together through les_ensemble_step, or one member after another."""

    def __init__(self, cases, device=None, share: int = 1, together: bool = True):
        """share > 1 caps every member's persistent CG solve at 1/share of the
        SMs (les_tuning.cg_max_blocks), so that up to `share` members solve
        at once; 1 leaves the solves uncapped (one at a time).  together:
        step the members concurrently (les_ensemble_step: a host thread per
        member, the members' kernels overlapping); False steps them one after
        another (tune() chooses by timing both)."""
        import torch
        self.torch = torch
        self.members = [Simulation(c, device=device, stream=torch.cuda.Stream(device=device)) for c in cases]
        self.lib = self.members[0].lib
        self.cells = sum(m.n for m in self.members)
        self.share = share
        self.together = together
        if share > 1:
            nsm = torch.cuda.get_device_properties(device if device is not None else
                                                   torch.cuda.current_device()).multi_processor_count
            for m in self.members:
                m.set_tuning(cg_max_blocks=max(1, nsm // share))

    def set_states(self, states) -> None:
        for m, st in zip(self.members, states):
            m.set_state(st)

    def step(self, nsteps: int = 1, allow_not_converged: bool = False) -> list:
        if not self.together:
            return [x.step(nsteps, allow_not_converged=allow_not_converged) for x in self.members]
        m = len(self.members)
        hs = (C.c_void_p * m)(*[x.h.value for x in self.members])
        stats = (LesStepStats * m)()
        failed = C.c_int32(-1)
        rc = self.lib.les_ensemble_step(hs, m, int(nsteps), stats, C.byref(failed))
        allow = (LES_OK, LES_ERR_NOT_CONVERGED) if allow_not_converged else (LES_OK,)
        if rc not in allow:
            h = self.members[failed.value].h if failed.value >= 0 else None
            _check(self.lib, h, rc, f"les_ensemble_step (member {failed.value})", allow)
        return [st.as_dict() for st in stats]

    def tune(self, steps: int = 2) -> dict:
        """Time `steps` ensemble steps stepped together and one member after
        another (after one untimed step each, L2 not flushed), from the same
        member states, keep the faster mode and put the states back.  On-chip
        solves are bound by the latency of their grid sums through L2, which
        the other members' streaming kernels raise when they run beside them;
        which mode wins depends on the members.  Returns {"together": chosen
        mode, "ms_per_step": {"together": ms, "one_after_another": ms}}."""
        import time
        torch = self.torch
        names = ("u", "v", "w", "p", "theta_l", "q_t")
        torch.cuda.synchronize()
        snaps = [{k: x.view(k).clone() for k in names} for x in self.members]
        dts = [x.dt for x in self.members]

        def restore():
            torch.cuda.synchronize()
            for x, snap, dt in zip(self.members, snaps, dts):
                for k in names:
                    x.view(k).copy_(snap[k])
                if dt:
                    x.dt = dt
            torch.cuda.synchronize()

        ms = {}
        for mode in (True, False):
            self.together = mode
            restore()
            self.step(1, allow_not_converged=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            self.step(steps, allow_not_converged=True)
            torch.cuda.synchronize()
            ms["together" if mode else "one_after_another"] = 1e3 * (time.perf_counter() - t0) / steps
        self.together = ms["together"] <= ms["one_after_another"]
        restore()
        return {"together": self.together, "ms_per_step": ms}

    def close(self) -> None:
        for x in self.members:
            x.close()


# candidate tunings for autotune(): the predictor kernels and, for the CG,
# the on-chip solver, its block cap, and the tiles of the streaming solver
AUTOTUNE_CANDIDATES = (
    {"stencil_path": 0},
    {"stencil_path": 1},
    {"stencil_path": 0, "cg_max_blocks": 64},
    {"stencil_path": 0, "cg_resident": 2},
    {"stencil_path": 0, "cg_resident": 1, "cg_variant": 2, "cg_tile_rows": 4, "cg_tile_planes": 4},
    {"stencil_path": 0, "cg_resident": 1, "cg_variant": 2, "cg_tile_rows": 2, "cg_tile_planes": 8},
    {"stencil_path": 0, "cg_resident": 1, "cg_variant": 3},
    {"stencil_path": 0, "cg_resident": 1, "cg_variant": 4},
)


def autotune(sim: "Simulation", candidates=AUTOTUNE_CANDIDATES, steps: int = 2) -> dict:
    """Time `steps` steps of the simulation under each candidate tuning (after
    one untimed step) from the same state, keep the fastest and put the state
    back.  Returns {"tuning": best candidate, "ms_per_step": {i: ms}}."""
    torch = sim.torch
    names = ("u", "v", "w", "p", "theta_l", "q_t")
    torch.cuda.synchronize()
    snap = {k: sim.view(k).clone() for k in names}
    base = sim.tuning()
    dt = sim.dt
    timings = {}

    def restore():
        torch.cuda.synchronize()
        for k in names:
            sim.view(k).copy_(snap[k])
        torch.cuda.synchronize()

    for i, cand in enumerate(candidates):
        t = dict(base)
        t.update(cand)
        sim.set_tuning(**t)
        restore()
        sim.step(1, allow_not_converged=True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(sim.stream)
        sim.step(steps, allow_not_converged=True)
        b.record(sim.stream)
        b.synchronize()
        timings[i] = a.elapsed_time(b) / steps
    best = min(timings, key=timings.get)
    t = dict(base)
    t.update(candidates[best])
    sim.set_tuning(**t)
    restore()
    if dt:
        sim.dt = dt
    return {"tuning": dict(candidates[best]), "ms_per_step": timings}
