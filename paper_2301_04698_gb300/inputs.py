"""Seeded synthetic workloads shared by the CUDA path and the CPU oracle.

This module describes *what* is simulated -- grid, spacings, switches,
parameter values and seeded initial fields -- and holds none of the method's
arithmetic: no reference state, thermodynamics, stencil or solver.  Both sides
convert a :class:`Case` into their own parameter structure.

Random numbers come from one counter-based generator: the SplitMix64 output
function (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to ``seed * golden + (stream << 40) + index``,
top 53 bits mapped to [0, 1).  Every draw is made here on the host; the GPU
never generates randomness.

Workloads (stand-ins for the paper's DYCOMS RF01 setup, Sec. 4, which needs
no external data beyond the printed parameters):

* ``tgv``   -- dry, triply periodic Taylor-Green box with unit reference
  density (the 32^3 FP64 parity case and its 1536x1536x256 tiling),
* ``cbl``   -- moist capped boundary layer: mixed layer of theta_l = 289 K,
  q_t = 9 g/kg (Sec. 4) below a seeded inversion height, seeded jumps above,
  +-0.1 K noise below, geostrophic wind, radiation, subsidence, surface
  fluxes and sponge.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_GOLD = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: physics switch names understood by both sides
PHYSICS = ("adv", "sgs", "const_nu", "moist", "buoy", "coriolis", "sponge",
           "rad", "subs", "sfc", "fb")

# stream ids of the generator
STREAM_U, STREAM_V, STREAM_W, STREAM_TH, STREAM_QT, STREAM_P = 0, 1, 2, 3, 4, 5
STREAM_CASE = 16
STREAM_ENSEMBLE = 17


def uniform01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from counter indices offset .. offset+n-1."""
    with np.errstate(over="ignore"):
        # (seed * golden + (stream << 40) + index) + golden, wrapping mod 2^64
        base = np.uint64(seed) * _GOLD + (np.uint64(stream) << np.uint64(40)) + _GOLD
        z = np.arange(offset, offset + n, dtype=np.uint64)
        z += base
        t = np.empty_like(z)
        np.right_shift(z, np.uint64(30), out=t)
        z ^= t
        z *= _M1
        np.right_shift(z, np.uint64(27), out=t)
        z ^= t
        z *= _M2
        np.right_shift(z, np.uint64(31), out=t)
        z ^= t
        z >>= np.uint64(11)
    out = z.astype(np.float64)
    out *= 1.0 / 9007199254740992.0
    return out


def uniform(seed: int, stream: int, n: int, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, stream, n, offset)


@dataclass
class Case:
    """A workload: grid, numerics switches, parameters and a seed."""

    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    walls: bool = False
    precision: int = 64
    dt: float = 0.0            # 0: Courant-number step from the initial field
    cfl: float = 0.3
    K: int = 3                 # sub-iterations per step
    solver: str = "cg"         # "cg" | "jacobi"
    op: str = "compact"        # "compact" (L_c + App. A term) | "wide" (D rho0 G)
    warm: str = "zero"         # "zero" | "prev" | "learned"
    tol: float = 1e-10
    maxit: int = 5000
    omega: float = 2.0 / 3.0
    solver_path: int = 0       # 0: persistent CG launch when eligible, 1: per-phase launches
    advection: str = "quick"   # "quick" | "weno3" (WENO3 with the local Lax-Friedrichs flux)
    precond: str = "none"      # "none" | "learned" (flexible CG with the network as preconditioner)
    physics: tuple = ("adv", "sgs")
    cs: float = 0.18
    pr: float = 0.4
    sc: float = 0.4
    nu_const: float = 0.0
    f_cor: float = 7.62e-5
    ug: float = 0.0
    vg: float = 0.0
    sponge_frac: float = 0.05
    sponge_rate: float = 0.25
    subs_div: float = 0.0
    shf: float = 0.0
    lhf: float = 0.0
    rad_f0: float = 0.0
    rad_f1: float = 0.0
    rad_kappa: float = 0.0
    theta0: float = 290.0
    p00: float = 1.0e5
    sat_tol: float = 1e-10
    sat_maxit: int = 20
    rho0_const: Optional[float] = None   # constant reference density override
    seed: int = 1
    init: str = "tgv"          # "tgv" | "cbl" | "zero"
    init_args: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self) -> tuple:
        return (self.nz, self.ny, self.nx)

    def replace(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)

    def rho0_profile(self) -> Optional[np.ndarray]:
        if self.rho0_const is None:
            return None
        return np.full(self.nz, float(self.rho0_const))


# ----------------------------------------------------------------------------
# case builders


def tgv(n: int = 32, nxyz: Optional[tuple] = None, seed: int = 1, precision: int = 64,
        cs: float = 0.17, amp: float = 1.0, noise: float = 1e-3, steps_tol: float = 1e-10,
        **kw) -> Case:
    """Dry triply periodic Taylor-Green box, dx = dy = dz = 1/n, rho0 = 1."""
    nx, ny, nz = nxyz if nxyz is not None else (n, n, n)
    h = 1.0 / n
    c = Case(name=f"tgv{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=h, dy=h, dz=h,
             walls=False, precision=precision, cfl=0.3, K=3, tol=steps_tol,
             physics=("adv", "sgs"), cs=cs, rho0_const=1.0, seed=seed,
             init="tgv", init_args={"amp": amp, "noise": noise, "theta": 300.0})
    return c.replace(**kw) if kw else c


def cbl(nx: int = 128, ny: int = 128, nz: int = 96, dx: float = 35.0, dz: float = 10.0,
        seed: int = 1, precision: int = 32, **kw) -> Case:
    """Moist capped boundary layer (DYCOMS RF01-like stand-in)."""
    c = Case(name=f"cbl{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, dz=dz,
             walls=True, precision=precision, dt=0.5, K=3, tol=1e-6, maxit=5000,
             physics=("adv", "sgs", "fb", "moist", "buoy", "coriolis", "sponge",
                      "rad", "subs", "sfc"),
             cs=0.18, pr=0.4, sc=0.4, f_cor=7.62e-5, ug=7.0, vg=-5.5,
             sponge_frac=0.05, sponge_rate=0.25, subs_div=3.75e-6,
             shf=15.0, lhf=115.0, rad_f0=70.0, rad_f1=22.0, rad_kappa=85.0,
             theta0=290.0, p00=1.0e5, sat_tol=1e-10 if precision == 64 else 1e-4,
             seed=seed, init="cbl",
             init_args={"theta_ml": 289.0, "qt_ml": 9.0e-3, "zi": (700.0, 900.0),
                        "dtheta": (5.0, 10.0), "dqt": (-8.0e-3, -5.0e-3),
                        "noise": 0.1})
    return c.replace(**kw) if kw else c


def density_current(dx: float = 200.0, ny: int = 4, precision: int = 64, **kw) -> Case:
    """Dry negatively buoyant bubble impinging on the surface (Sec. 3,
    density current): a -15 K perturbation of radii 4 km (horizontal) and
    2 km (vertical) in a uniform 300 K potential temperature, 51.2 km x 6.4
    km, periodic in x, uniform kinematic viscosity 10 m^2/s.  Two-dimensional
    as a thin periodic y extent with y-independent fields.  Readings (the
    paper does not state them): centre at mid-domain, 3 km up; cosine-squared
    bell; scalar diffusivity equal to the viscosity; the walls of the solver
    (free-slip surface, no-slip lid); a fixed step of dx / 200 s."""
    nx, nz = int(round(51200.0 / dx)), int(round(6400.0 / dx))
    c = Case(name=f"density_current{dx:g}m", nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, dz=dx, walls=True,
             precision=precision, dt=dx / 200.0, K=3, tol=1e-10 if precision == 64 else 1e-6,
             maxit=20000, physics=("adv", "const_nu", "buoy"), nu_const=10.0, pr=1.0, sc=1.0,
             theta0=300.0, init="bubble",
             init_args={"theta": 300.0, "amp": -15.0, "xc": 25600.0, "zc": 3000.0, "xr": 4000.0, "zr": 2000.0})
    return c.replace(**kw) if kw else c


def rising_bubble(dx: float = 200.0, ny: int = 4, precision: int = 64, **kw) -> Case:
    """Dry warm bubble (Sec. 3, rising bubble): a +2 K perturbation in a
    uniform 300 K potential temperature, 20 km x 10 km, periodic in x,
    uniform kinematic viscosity 1 m^2/s.  Readings: radius 2 km, centre at
    mid-domain, 2 km up; cosine-squared bell; otherwise as the density
    current."""
    nx, nz = int(round(20000.0 / dx)), int(round(10000.0 / dx))
    c = Case(name=f"rising_bubble{dx:g}m", nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, dz=dx, walls=True,
             precision=precision, dt=dx / 200.0, K=3, tol=1e-10 if precision == 64 else 1e-6,
             maxit=20000, physics=("adv", "const_nu", "buoy"), nu_const=1.0, pr=1.0, sc=1.0,
             theta0=300.0, init="bubble",
             init_args={"theta": 300.0, "amp": 2.0, "xc": 10000.0, "zc": 2000.0, "xr": 2000.0, "zr": 2000.0})
    return c.replace(**kw) if kw else c


def bubble_perturbation(case: Case) -> np.ndarray:
    """theta' of a bubble case on the nodes, (nz, ny, nx): amp cos^2(pi L / 2)
    for L <= 1, L the distance from the centre in units of the radii."""
    a = case.init_args
    x = (np.arange(case.nx) + 0.5) * case.dx
    z = (np.arange(case.nz) + 0.5) * case.dz
    L = np.sqrt(((x[None, :] - a["xc"]) / a["xr"]) ** 2 + ((z[:, None] - a["zc"]) / a["zr"]) ** 2)
    th = np.where(L <= 1.0, a["amp"] * np.cos(0.5 * np.pi * np.minimum(L, 1.0)) ** 2, 0.0)
    return np.broadcast_to(th[:, None, :], case.shape).copy()


# ----------------------------------------------------------------------------
# initial fields


def cbl_draws(case: Case) -> dict:
    """The seeded scalars of a capped-boundary-layer member."""
    a = case.init_args
    r = uniform01(case.seed, STREAM_CASE, 3)
    zi = a["zi"][0] + (a["zi"][1] - a["zi"][0]) * r[0]
    dth = a["dtheta"][0] + (a["dtheta"][1] - a["dtheta"][0]) * r[1]
    dq = a["dqt"][0] + (a["dqt"][1] - a["dqt"][0]) * r[2]
    return {"zi": float(zi), "dtheta": float(dth), "dqt": float(dq)}


def initial_state(case: Case) -> dict:
    """Seeded initial fields u, v, w, p, theta_l, q_t as float64 (nz, ny, nx)."""
    nz, ny, nx = case.shape
    n = case.n
    out = {}
    if case.init == "tgv":
        a = case.init_args
        x = (np.arange(nx) + 0.5) * case.dx
        y = (np.arange(ny) + 0.5) * case.dy
        z = (np.arange(nz) + 0.5) * case.dz
        tp = 2.0 * np.pi
        amp, eps = a.get("amp", 1.0), a.get("noise", 1e-3)
        sx, cx = np.sin(tp * x)[None, None, :], np.cos(tp * x)[None, None, :]
        sy, cy = np.sin(tp * y)[None, :, None], np.cos(tp * y)[None, :, None]
        cz = np.cos(tp * z)[:, None, None]
        for k in ("u", "v", "w"):
            out[k] = np.empty(case.shape)
        # plane chunks keep the temporaries small on large grids; the values
        # are those of the whole-array expressions
        plane = nx * ny
        step = max(1, (1 << 24) // plane)
        for k0 in range(0, nz, step):
            k1 = min(nz, k0 + step)
            m = (k1 - k0) * plane
            zs = slice(k0, k1)
            out["u"][zs] = amp * sx * cy * cz[zs] + \
                uniform(case.seed, STREAM_U, m, -eps, eps, offset=k0 * plane).reshape(k1 - k0, ny, nx)
            out["v"][zs] = -amp * cx * sy * cz[zs] + \
                uniform(case.seed, STREAM_V, m, -eps, eps, offset=k0 * plane).reshape(k1 - k0, ny, nx)
            out["w"][zs] = 0.0 + \
                uniform(case.seed, STREAM_W, m, -eps, eps, offset=k0 * plane).reshape(k1 - k0, ny, nx)
        out["theta_l"] = np.full(case.shape, a.get("theta", 300.0))
        out["q_t"] = np.zeros(case.shape)
    elif case.init == "cbl":
        a = case.init_args
        d = cbl_draws(case)
        z = (np.arange(nz) + 0.5) * case.dz
        below = (z < d["zi"])[:, None, None] * np.ones(case.shape, dtype=bool)
        th = np.where(below, a["theta_ml"], a["theta_ml"] + d["dtheta"])
        qt = np.where(below, a["qt_ml"], a["qt_ml"] + d["dqt"])
        noise = uniform(case.seed, STREAM_TH, n, -a["noise"], a["noise"]).reshape(case.shape)
        out["theta_l"] = th + np.where(below, noise, 0.0)
        out["q_t"] = qt.astype(np.float64)
        out["u"] = np.full(case.shape, case.ug)
        out["v"] = np.full(case.shape, case.vg)
        out["w"] = np.zeros(case.shape)
    elif case.init == "bubble":
        out["theta_l"] = case.init_args["theta"] + bubble_perturbation(case)
        for k in ("u", "v", "w", "q_t"):
            out[k] = np.zeros(case.shape)
    elif case.init == "zero":
        for k in ("u", "v", "w", "theta_l", "q_t"):
            out[k] = np.zeros(case.shape)
    else:
        raise ValueError(f"unknown init {case.init!r}")
    out["p"] = np.zeros(case.shape)
    return out


def ensemble(m: int = 16, seed: int = 1, xy=(64, 96, 128, 160, 192), zs=(64, 96, 128),
             precision: int = 32) -> list:
    """Members of an uneven ensemble of capped boundary layers: member i draws
    its horizontal size from `xy`, its height from `zs`, its own inversion
    (the cbl seed), and scales of the surface fluxes and of the subsidence
    divergence in [0.5, 1.5) -- all from the counter generator."""
    out = []
    for i in range(m):
        r = uniform01(seed, STREAM_ENSEMBLE, 5, offset=5 * i)
        n = xy[int(r[0] * len(xy)) % len(xy)]
        nz = zs[int(r[1] * len(zs)) % len(zs)]
        c = cbl(n, n, nz, seed=1000 * seed + i, precision=precision)
        out.append(c.replace(name=f"member{i}_{n}x{n}x{nz}", shf=c.shf * (0.5 + r[2]),
                             lhf=c.lhf * (0.5 + r[3]), subs_div=c.subs_div * (0.5 + r[4])))
    return out
