"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed-form
amplification factor of a Fourier mode, an FFT / DCT solve, an exact budget, a
telescoping identity or a brute-force root.  The constructions are chosen so
that a dropped term, a wrong sign, a wrong index or a transposed operand in the
oracle fails at least one of them.
"""
import numpy as np
import pytest
import scipy.fft as sfft

from paper_2301_04698_gb300 import inputs
from oracle import Oracle


def _grid(c):
    x = (np.arange(c.nx) + 0.5) * c.dx
    y = (np.arange(c.ny) + 0.5) * c.dy
    z = (np.arange(c.nz) + 0.5) * c.dz
    return np.meshgrid(z, y, x, indexing="ij")


def _base(nx, ny, nz, h=1.0, walls=False, physics=(), **kw):
    c = inputs.Case(name="pin", nx=nx, ny=ny, nz=nz, dx=h, dy=h, dz=h, walls=walls,
                    precision=64, physics=tuple(physics), rho0_const=1.0, init="zero",
                    tol=1e-13, maxit=20000)
    return c.replace(**kw)


def _gk(z, K):
    """Amplification of the K-sub-iteration scheme for du/dt = lambda u, z = lambda dt:
    phi^{k+1} = phi^n + dt lambda (phi^k + phi^n) / 2, phi^0 = phi^n (Sec. 2.4)."""
    g = 1.0 + 0.0j
    for _ in range(K):
        g = 1.0 + 0.5 * z * (g + 1.0)
    return g


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# --------------------------------------------------------------------------
# QUICK advection + iterative time scheme: sine translation, both upwind branches


@pytest.mark.parametrize("u0", [0.7, -0.55])
@pytest.mark.parametrize("K", [1, 3])
def test_quick_translation_closed_form(u0, K):
    n, m, steps = 32, 3, 20
    c = _base(n, 4, 4, h=1.0 / n, physics=("adv",), K=K, dt=0.3 / n / abs(u0))
    Z, Y, X = _grid(c)
    th = 300.0 + np.sin(2 * np.pi * m * X)
    o = Oracle(c, {"u": np.full(c.shape, u0), "v": np.zeros(c.shape), "w": np.zeros(c.shape),
                   "theta_l": th, "q_t": np.zeros(c.shape)})
    o.step(steps)
    th_ang = 2 * np.pi * m / n
    cth = np.cos(th_ang)
    # semi-discrete QUICK symbol: lambda = -|u|/dx (1-cos)^2/4 - i u/dx (10 sin - sin 2)/8
    lam = -abs(u0) / c.dx * (1 - cth) ** 2 / 4 - 1j * u0 / c.dx * (10 * np.sin(th_ang) - np.sin(2 * th_ang)) / 8
    G = _gk(lam * c.dt, K) ** steps
    i = np.arange(n)
    expect_row = np.imag(G * np.exp(1j * th_ang * (i + 0.5) * n * c.dx))
    got = o.get("theta_l") - 300.0
    assert np.max(np.abs(got - expect_row[None, None, :])) < 1e-12
    # the uniform velocity is an exact steady state of the momentum update
    assert np.max(np.abs(o.get("u") - u0)) < 1e-13


# --------------------------------------------------------------------------
# WENO3 with the local Lax-Friedrichs flux (the alternative advection scheme)


def _x_profile(c, prof):
    x = (np.arange(c.nx) + 0.5) / c.nx
    return prof(x)[None, None, :] * np.ones(c.shape)


def _advect(scheme, n, prof, u0=0.7, K=3, steps=None, T=None):
    c = _base(n, 4, 4, h=1.0 / n, physics=("adv",), K=K, dt=0.3 / n / abs(u0), advection=scheme)
    o = Oracle(c, {"u": np.full(c.shape, u0), "v": np.zeros(c.shape), "w": np.zeros(c.shape),
                   "theta_l": _x_profile(c, prof), "q_t": np.zeros(c.shape)})
    steps = steps if steps is not None else int(round(T / c.dt))
    o.step(steps)
    return c, o.get("theta_l"), steps


@pytest.mark.parametrize("u0", [0.7, -0.55])
def test_weno3_smooth_limit_closed_form(u0):
    """For a smooth wave of small amplitude on a large mean the smoothness
    indicators are far below eps, the weights take their ideal values 1/3, 2/3
    and the face value is the linear third-order upwind-biased one,
    (-phi_{n-1} + 5 phi_n + 2 phi_{n+1}) / 6 (mirrored for u < 0): the mode
    follows that symbol through the K-sub-iteration scheme."""
    n, m, steps, K, A = 32, 3, 20, 3, 1e-4
    c, th, _ = _advect("weno3", n, lambda x: 300.0 + A * np.sin(2 * np.pi * m * x), u0=u0, K=K, steps=steps)
    t = 2 * np.pi * m / n
    e = np.exp(1j * t)
    face = (-1 / e + 5 + 2 * e) / 6 if u0 > 0 else (2 + 5 * e - e * e) / 6
    lam = -u0 / c.dx * face * (1 - 1 / e)
    G = _gk(lam * c.dt, K) ** steps
    i = np.arange(n)
    expect = A * np.imag(G * np.exp(1j * t * (i + 0.5)))
    assert np.max(np.abs(th[0, 0] - 300.0 - expect)) < 1e-9


def test_weno3_square_wave_is_nearly_non_oscillatory():
    """A translated step: WENO3 creates far smaller new extrema than QUICK
    (QUICK is linear and third order, so it overshoots by ~13 % here)."""
    prof = lambda x: 300.0 + ((x > 0.25) & (x < 0.5)) * 1.0
    over = {}
    for s in ("quick", "weno3"):
        _, th, _ = _advect(s, 64, prof, steps=40)
        over[s] = max(th.max() - 301.0, 300.0 - th.min())
    assert over["quick"] > 0.08
    assert over["weno3"] < 0.05 and over["weno3"] < 0.3 * over["quick"]


def test_weno3_self_convergence():
    """Smooth translation with the nonlinear weights active (amplitude 1): the
    error against the exact translated wave falls at least 4x per halving of
    the spacing at fixed Courant number."""
    errs = []
    for n in (32, 64, 128):
        c, th, steps = _advect("weno3", n, lambda x: 300.0 + np.sin(2 * np.pi * x), T=0.5)
        x = (np.arange(n) + 0.5) / n
        exact = 300.0 + np.sin(2 * np.pi * (x - 0.7 * steps * c.dt))
        errs.append(np.sqrt(np.mean((th[0, 0] - exact) ** 2)))
    assert errs[0] / errs[1] > 4.0 and errs[1] / errs[2] > 4.0


# --------------------------------------------------------------------------
# 2nd-order central diffusion of scalars, Pr for theta_l and Sc for q_t


def test_scalar_diffusion_closed_form():
    nx, ny, nz = 12, 10, 8
    nu, pr, sc, steps, K = 0.01, 0.4, 0.7, 5, 3
    c = _base(nx, ny, nz, h=0.1, physics=("const_nu",), nu_const=nu, pr=pr, sc=sc, K=K, dt=0.05,
              dx=0.1, dy=0.13, dz=0.07)
    Z, Y, X = _grid(c)
    th_ang = [2 * np.pi * 1 / nx, 2 * np.pi * 2 / ny, 2 * np.pi * 1 / nz]
    Ls = [nx * c.dx, ny * c.dy, nz * c.dz]
    mode = (np.sin(2 * np.pi * 1 * X / Ls[0]) * np.sin(2 * np.pi * 2 * Y / Ls[1]) *
            np.cos(2 * np.pi * 1 * Z / Ls[2]))
    o = Oracle(c, {"theta_l": 290 + mode, "q_t": 0.01 * mode})
    o.step(steps)
    hs = [c.dx, c.dy, c.dz]
    sym = -sum(4.0 / h ** 2 * np.sin(t / 2) ** 2 for t, h in zip(th_ang, hs))
    Gth = _gk(sym * nu / pr * c.dt, K).real ** steps
    Gq = _gk(sym * nu / sc * c.dt, K).real ** steps
    assert np.max(np.abs(o.get("theta_l") - 290 - Gth * mode)) < 1e-12
    assert np.max(np.abs(o.get("q_t") - 0.01 * Gq * mode)) < 1e-14


# --------------------------------------------------------------------------
# Stokes Taylor-Green vortex: SGS stress divergence with its cross terms


def test_stokes_tgv_closed_form():
    n, nu, steps, K = 16, 0.05, 4, 3
    h = 1.0 / n
    c = _base(n, n, n, h=h, physics=("const_nu",), nu_const=nu, K=K, dt=0.2 * h * h / nu)
    Z, Y, X = _grid(c)
    tp = 2 * np.pi
    u = np.sin(tp * X) * np.cos(tp * Y) * np.cos(tp * Z)
    v = -np.cos(tp * X) * np.sin(tp * Y) * np.cos(tp * Z)
    o = Oracle(c, {"u": u, "v": v, "w": np.zeros(c.shape)})
    o.step(steps)
    s2 = np.sin(tp / n / 2) ** 2
    # div(nu (grad u + grad u^T)) on this mode: -nu (4 s2 / h^2) (3 + s2)
    mu = -nu * (4 * s2 / h ** 2) * (3 + s2)
    G = _gk(mu * c.dt, K).real ** steps
    assert np.max(np.abs(o.get("u") - G * u)) < 1e-12
    assert np.max(np.abs(o.get("v") - G * v)) < 1e-12
    assert np.max(np.abs(o.get("w"))) < 1e-12


# --------------------------------------------------------------------------
# Coriolis: inertial oscillation of a uniform current


def test_coriolis_inertial_oscillation():
    f, dt, steps, K = 1e-3, 40.0, 7, 3
    c = _base(6, 5, 4, h=10.0, physics=("coriolis",), f_cor=f, K=K, dt=dt)
    U, V = 3.0, -1.5
    o = Oracle(c, {"u": np.full(c.shape, U), "v": np.full(c.shape, V)})
    o.step(steps)
    Wc = _gk(-1j * f * dt, K) ** steps * (U + 1j * V)
    assert np.max(np.abs(o.get("u") - Wc.real)) < 1e-12
    assert np.max(np.abs(o.get("v") - Wc.imag)) < 1e-12


# --------------------------------------------------------------------------
# Sponge: Rayleigh damping per level, zero below the sponge base


def test_sponge_damping_per_level():
    nz, dt, steps, K, rate, frac = 40, 0.5, 3, 3, 0.25, 0.2
    c = _base(4, 4, nz, h=10.0, walls=True, physics=("sponge",), sponge_rate=rate,
              sponge_frac=frac, ug=0.0, vg=0.0, K=K, dt=dt)
    o = Oracle(c, {"u": np.full(c.shape, 2.0), "v": np.full(c.shape, -1.0)})
    o.step(steps)
    z = (np.arange(nz) + 0.5) * c.dz
    H = nz * c.dz
    zs = (1 - frac) * H
    beta = np.where(z > zs, rate * np.sin(0.5 * np.pi * (z - zs) / (H - zs)) ** 2, 0.0)
    G = np.array([_gk(-b * dt, K).real ** steps for b in beta])
    u = o.get("u")[:, 0, 0]
    assert np.max(np.abs(u - 2.0 * G)) < 1e-12
    assert np.all(u[z <= zs] == 2.0)
    assert np.all(np.diff(u[z > zs]) < 0)   # stronger damping toward the lid


# --------------------------------------------------------------------------
# Poisson operator and solvers against FFT / DCT solves


def _poisson_fft(b, c):
    nz, ny, nx = b.shape
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    lam_x = -4 / c.dx ** 2 * np.sin(kx / 2) ** 2
    lam_y = -4 / c.dy ** 2 * np.sin(ky / 2) ** 2
    if c.walls:
        m = np.arange(nz)
        lam_z = -4 / c.dz ** 2 * np.sin(np.pi * m / (2 * nz)) ** 2
        bh = sfft.dct(np.fft.fft2(b, axes=(1, 2)), type=2, axis=0, norm="ortho")
    else:
        kz = 2 * np.pi * np.fft.fftfreq(nz)
        lam_z = -4 / c.dz ** 2 * np.sin(kz / 2) ** 2
        bh = np.fft.fftn(b)
    lam = lam_z[:, None, None] + lam_y[None, :, None] + lam_x[None, None, :]
    lam[0, 0, 0] = 1.0
    xh = bh / lam
    xh[0, 0, 0] = 0.0
    if c.walls:
        x = np.fft.ifft2(sfft.idct(xh, type=2, axis=0, norm="ortho"), axes=(1, 2)).real
    else:
        x = np.fft.ifftn(xh).real
    return x


@pytest.mark.parametrize("walls", [False, True])
def test_poisson_cg_matches_fft(walls):
    c = _base(12, 10, 9, walls=walls, dx=0.3, dy=0.25, dz=0.1)
    o = Oracle(c)
    b = inputs.uniform(7, 0, c.n, -1, 1).reshape(c.shape)
    b -= b.mean()
    x, st, it, res = o.poisson(b, tol=1e-13, maxit=5000)
    assert st == 0 and res <= 1e-13
    ref = _poisson_fft(b, c)
    assert _rel(x, ref) < 1e-10
    assert abs(x.mean()) < 1e-14
    # the operator itself, on a smooth field
    y = o.apply_poisson(ref)
    assert _rel(y, b) < 1e-11


def test_poisson_jacobi_matches_fft():
    c = _base(8, 6, 6, walls=True, dx=0.3, dy=0.3, dz=0.2, omega=2.0 / 3.0)
    o = Oracle(c)
    b = inputs.uniform(3, 0, c.n, -1, 1).reshape(c.shape)
    b -= b.mean()
    x, st, it, res = o.poisson(b, solver="jacobi", tol=1e-9, maxit=200000)
    assert st == 0 and it > 10
    assert _rel(x, _poisson_fft(b, c)) < 1e-7


def test_poisson_rhs_mean_is_removed():
    c = _base(8, 8, 8)
    o = Oracle(c)
    b = inputs.uniform(5, 0, c.n, -1, 1).reshape(c.shape)
    x1, *_ = o.poisson(b, tol=1e-12)
    x2, *_ = o.poisson(b - b.mean(), tol=1e-12)
    assert np.max(np.abs(x1 - x2)) < 1e-12


# --------------------------------------------------------------------------
# Appendix A: C = (L_w - L_c) psi, symbol +4 sin^4(theta/2) / Delta^2 per direction


@pytest.mark.parametrize("walls", [False, True])
def test_appendix_a_correction_symbol(walls):
    c = _base(12, 10, 8, walls=walls, dx=0.3, dy=0.2, dz=0.1, dt=0.5)
    o = Oracle(c)
    psi = inputs.uniform(11, 0, c.n, -1, 1).reshape(c.shape)
    o.begin_step()
    o.set("psi", psi)
    o.momentum_stage()
    rhs = o.get("rhs")
    nz, ny, nx = c.shape
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    cx = 4 / c.dx ** 2 * np.sin(kx / 2) ** 4
    cy = 4 / c.dy ** 2 * np.sin(ky / 2) ** 4
    if walls:
        th = np.pi * np.arange(nz) / nz
        cz = 4 / c.dz ** 2 * np.sin(th / 2) ** 4
        ph = sfft.dct(np.fft.fft2(psi, axes=(1, 2)), type=2, axis=0, norm="ortho")
        sym = cz[:, None, None] + cy[None, :, None] + cx[None, None, :]
        Cpsi = np.fft.ifft2(sfft.idct(sym * ph, type=2, axis=0, norm="ortho"), axes=(1, 2)).real
    else:
        kz = 2 * np.pi * np.fft.fftfreq(nz)
        cz = 4 / c.dz ** 2 * np.sin(kz / 2) ** 4
        sym = cz[:, None, None] + cy[None, :, None] + cx[None, None, :]
        Cpsi = np.fft.ifftn(sym * np.fft.fftn(psi)).real
    # rhs = alpha0 / dt D(rho0 u^) - C, and u^ = 0 here
    assert np.max(np.abs(rhs + Cpsi)) < 1e-10 * np.max(np.abs(Cpsi))


# --------------------------------------------------------------------------
# consistent projection: D(rho0 u) vanishes after the D(rho0 G) solve


def test_wide_projection_is_divergence_free():
    n = 16
    c = _base(n, n, n, h=1.0 / n, physics=(), op="wide", K=1, dt=0.01, tol=1e-14, maxit=5000)
    u = {k: inputs.uniform(2, s, c.n, -1, 1).reshape(c.shape) for k, s in (("u", 0), ("v", 1), ("w", 2))}
    o = Oracle(c, u)
    before = o.diagnostics()["max_div"]
    o.begin_step()
    o.momentum_stage()
    st, it, res = o.solve_stage()
    o.correct_stage()
    after = o.diagnostics()["max_div"]
    assert before > 10.0
    assert after < 1e-10


# --------------------------------------------------------------------------
# conservation (Sec. 2.4: exact discrete conservation without sources)


@pytest.mark.parametrize("walls,advection", [(False, "quick"), (True, "quick"), (False, "weno3"),
                                             (True, "weno3")])
def test_scalar_and_momentum_conservation(walls, advection):
    c = _base(10, 8, 8, h=0.1, walls=walls, physics=("adv", "sgs"), cs=0.3, dt=0.02, K=3,
              tol=1e-12, dx=0.1, dy=0.12, dz=0.08, advection=advection)
    if walls:
        c = c.replace(rho0_const=None, dz=25.0, dx=40.0, dy=40.0, dt=0.5)
    st = {k: inputs.uniform(4, s, c.n, -1, 1).reshape(c.shape) for k, s in (("u", 0), ("v", 1), ("w", 2))}
    st["theta_l"] = 290 + inputs.uniform(4, 3, c.n, -2, 2).reshape(c.shape)
    st["q_t"] = 0.01 + inputs.uniform(4, 4, c.n, -2e-3, 2e-3).reshape(c.shape)
    o = Oracle(c, st)
    d0 = o.diagnostics()
    o.step(4)
    d1 = o.diagnostics()
    assert abs(d1["sum_rho_theta"] - d0["sum_rho_theta"]) <= 1e-13 * abs(d0["sum_rho_theta"])
    assert abs(d1["sum_rho_qt"] - d0["sum_rho_qt"]) <= 1e-13 * abs(d0["sum_rho_qt"])
    if not walls:
        for k in ("sum_rho_u", "sum_rho_v", "sum_rho_w"):
            assert abs(d1[k] - d0[k]) < 1e-12


# --------------------------------------------------------------------------
# surface fluxes, subsidence and radiation: budgets and exact profiles


def test_surface_flux_budget():
    c = _base(6, 5, 8, walls=True, physics=("sfc",), shf=15.0, lhf=115.0, dt=2.0, K=3,
              dx=35.0, dy=35.0, dz=10.0, rho0_const=None)
    o = Oracle(c, {"theta_l": np.full(c.shape, 289.0), "q_t": np.full(c.shape, 9e-3)})
    d0 = o.diagnostics()
    o.step(3)
    d1 = o.diagnostics()
    area = c.nx * c.dx * c.ny * c.dy
    # SHF / c_pd and LHF / L_v0 enter through the surface face every step
    tol_th = 1e-13 * d0["sum_rho_theta"]
    tol_q = 1e-13 * d0["sum_rho_qt"]
    assert abs(d1["sum_rho_theta"] - d0["sum_rho_theta"] - 3 * 2.0 * 15.0 / 1004.5 * area) < tol_th
    assert abs(d1["sum_rho_qt"] - d0["sum_rho_qt"] - 3 * 2.0 * 115.0 / 2.47e6 * area) < tol_q


def test_subsidence_upwind_from_above():
    D, dt = 3.75e-6, 5.0
    c = _base(3, 3, 20, walls=True, physics=("subs",), subs_div=D, dt=dt, K=1, dz=10.0,
              dx=10.0, dy=10.0)
    z = (np.arange(c.nz) + 0.5) * c.dz
    th = 290 + 1e-4 * z ** 2
    o = Oracle(c, {"theta_l": np.broadcast_to(th[:, None, None], c.shape).copy()})
    o.step(1)
    got = o.get("theta_l")[:, 1, 1]
    # sinking air carries theta_l down: the derivative is taken from the level above
    up = 1e-4 * ((z + c.dz) ** 2 - z ** 2) / c.dz
    expect = th + dt * D * z * up
    expect[-1] = th[-1]              # mirror ghost above the top node
    assert np.max(np.abs(got - expect)) < 1e-12


def test_radiation_column_telescopes():
    c = inputs.cbl(4, 3, 40, dz=25.0, precision=64).replace(
        physics=("moist", "rad"), dt=1.0, K=1)
    st = inputs.initial_state(c)
    o = Oracle(c, st)
    o.begin_step()
    ql = o.get("q_l")
    srad = o.get("s_rad")
    T = o.get("T")
    rho0, p0 = o.profiles()
    qt = st["q_t"]
    cpm = (1 - qt) * 1004.5 + (qt - ql) * 1859.5 + ql * 4181.0
    Rm = (1 - qt) * 287.0 + (qt - ql) * 461.89
    Pi = (p0[:, None, None] / 1e5) ** (Rm / cpm)
    lwp = (rho0[:, None, None] * ql * c.dz).sum(axis=0)
    assert np.all(lwp > 0)
    F_top = c.rad_f0 + c.rad_f1 * np.exp(-c.rad_kappa * lwp)
    F_bot = c.rad_f0 * np.exp(-c.rad_kappa * lwp) + c.rad_f1
    col = (srad * cpm * Pi * c.dz).sum(axis=0)
    assert np.max(np.abs(col + (F_top - F_bot))) < 1e-9
    # cloud-top cooling dominates: the net column heating is negative
    assert np.all(col < 0)
    # levels far below the cloud see no flux divergence
    assert np.all(srad[:3][ql[:3] == 0] == 0.0) or np.max(np.abs(srad[:3])) < 1e-9
    assert np.all(np.isfinite(T))


# --------------------------------------------------------------------------
# thermodynamics (Sec. 2.1-2.2)


def test_reference_state_hydrostatic():
    c = inputs.cbl(4, 4, 200, dz=5.0, precision=64)
    o = Oracle(c)
    rho0, p0 = o.profiles()
    z = (np.arange(c.nz) + 0.5) * c.dz
    dpdz = (p0[2:] - p0[:-2]) / (2 * c.dz)
    assert np.max(np.abs(dpdz + rho0[1:-1] * 9.81) / (rho0[1:-1] * 9.81)) < 1e-6
    # extrapolating to the surface gives p00
    p_s = p0[0] + (p0[0] - p0[1]) * 0.5
    assert abs(p_s - c.p00) / c.p00 < 1e-6


def test_saturation_adjustment():
    c = inputs.cbl(4, 4, 96, precision=64)
    o = Oracle(c)
    rho0, p0 = o.profiles()
    # unsaturated: T = Pi theta_l exactly, q_l = 0
    T, ql = o.saturation(0, 300.0, 1e-3)
    assert ql == 0.0
    assert T == pytest.approx(300.0 * (p0[0] / 1e5) ** (((1 - 1e-3) * 287 + 1e-3 * 461.89) /
                                                       ((1 - 1e-3) * 1004.5 + 1e-3 * 1859.5)),
                              rel=1e-15)
    # dry limit
    T, ql = o.saturation(50, 290.0, 0.0)
    assert ql == 0.0 and T == pytest.approx(290.0 * (p0[50] / 1e5) ** (287 / 1004.5), rel=1e-15)
    # saturated: the secant root solves theta_l*(T) = theta_l, and agrees with bisection
    for k, th, qt in ((80, 289.0, 9e-3), (60, 289.5, 1.2e-2), (90, 288.0, 1.5e-2)):
        T, ql = o.saturation(k, th, qt)
        assert ql > 0
        assert abs(o.theta_l_star(k, T, qt) - th) < 1e-10
        assert ql == pytest.approx(qt - o.qv_star(k, T), rel=1e-12)
        lo, hi = 200.0, 330.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if o.theta_l_star(k, mid, qt) < th:
                lo = mid
            else:
                hi = mid
        assert abs(T - 0.5 * (lo + hi)) < 1e-8
    # theta_l* is monotone in T (unique root)
    Ts = np.linspace(250, 320, 400)
    f = np.array([o.theta_l_star(70, t, 9e-3) for t in Ts])
    assert np.all(np.diff(f) > 0)
    # q_v* at the triple point reduces to the vapour pressure e_tr
    eps = 287.0 / 461.89
    assert o.qv_star(0, 273.16) == pytest.approx(eps * 611.657 / (p0[0] - (1 - eps) * 611.657), rel=1e-14)


def test_buoyancy_vanishes_in_the_reference_state():
    c = inputs.cbl(4, 4, 50, precision=64).replace(physics=("buoy",), dt=1.0)
    o = Oracle(c, {"theta_l": np.full(c.shape, c.theta0), "q_t": np.zeros(c.shape)})
    o.begin_step()
    assert np.max(np.abs(o.get("b"))) < 1e-12
    o2 = Oracle(c, {"theta_l": np.full(c.shape, c.theta0 + 1.0), "q_t": np.zeros(c.shape)})
    o2.begin_step()
    b = o2.get("b")
    # a warmer parcel is buoyant by about g dtheta / theta0
    assert np.all(b > 0) and np.allclose(b, 9.81 / c.theta0, rtol=2e-2)


# --------------------------------------------------------------------------
# Smagorinsky viscosity (Sec. 2.3)


def test_smagorinsky_shear_closed_form():
    n = 16
    c = _base(4, n, 4, h=1.0 / n, physics=("sgs",), cs=0.17)
    Z, Y, X = _grid(c)
    u = np.sin(2 * np.pi * Y)
    o = Oracle(c)
    nu = o.nu_field(u, np.zeros(c.shape), np.zeros(c.shape), np.zeros(c.shape))
    dudy = np.sin(2 * np.pi / n) / c.dy * np.cos(2 * np.pi * Y)
    assert np.max(np.abs(nu - (0.17 * c.dx) ** 2 * np.abs(dudy))) < 1e-14


def test_buoyancy_factor_limits_mixing():
    n, N2 = 16, 2e-4
    c = _base(4, n, 12, h=1.0 / n, walls=True, physics=("sgs", "fb"), cs=0.17, pr=0.4,
              dx=1.0, dy=1.0, dz=1.0)
    Z, Y, X = _grid(c)
    u = np.sin(2 * np.pi * Y / n) * 0.01 * n
    b = N2 * Z
    o = Oracle(c)
    nu = o.nu_field(u, np.zeros(c.shape), np.zeros(c.shape), b)
    S = np.abs(np.sin(2 * np.pi / n) * 0.01 * n * np.cos(2 * np.pi * Y / n))   # = sqrt(2 S_ij S_ij)
    with np.errstate(divide="ignore", invalid="ignore"):
        fb = np.sqrt(np.clip(1 - N2 / (0.4 * S ** 2), 0, 1))
    expect = 0.17 ** 2 * fb * S
    inner = slice(1, -1)
    assert np.max(np.abs(nu[inner] - expect[inner])) < 1e-14
    assert np.all(nu[inner] <= 0.17 ** 2 * S[inner] + 1e-15)
    # the no-slip lid adds shear at the top node (u ghost = -u)
    assert np.all(nu[-1] > nu[-2])


# --------------------------------------------------------------------------
# Taylor-Green with Smagorinsky: kinetic energy does not grow


def test_tgv_energy_decays():
    c = inputs.tgv(16)
    o = Oracle(c, inputs.initial_state(c))
    e = [o.diagnostics()["kinetic_energy"]]
    for _ in range(4):
        o.step(1)
        e.append(o.diagnostics()["kinetic_energy"])
    assert all(b < a for a, b in zip(e, e[1:]))
