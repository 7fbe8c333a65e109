"""Pins of the oracle's momentum stage (Sec. 2.4, Eq. momentum_prediction_step).

The momentum predictor is
    rho0 u^ = rho0 u^n + dt [ -rho0 G(alpha0 p^k) + R(u^{n+1/2}) ],
    R = -div(rho0 u^{n+1/2} (x) u^{n+1/2}) + div(rho0 2 nu_t S) + rho0 b k
        - f k x rho0 (u^{n+1/2} - u_g) - sponge,
with u^{n+1/2} = (u^k + u^n) / 2.  Each test below fixes one group of its
terms against mathematics that does not go through the oracle's stencils:
the Fourier symbol of QUICK carried through the sub-iteration recurrence, an
exact discrete rest state, the continuum dissipation of the Smagorinsky
model and its exact continuum force.  Each docstring names the slips it
rules out; each named slip, planted in a copy of the oracle, fails its test.
"""
import numpy as np
import pytest

from paper_2301_04698_gb300 import inputs
from oracle import Oracle


def _case(nx, ny, nz, h, walls=False, physics=(), rho0_const=1.0, **kw):
    c = inputs.Case(name="mpin", nx=nx, ny=ny, nz=nz, dx=h, dy=h, dz=h, walls=walls, precision=64,
                    physics=tuple(physics), rho0_const=rho0_const, init="zero", tol=1e-13, maxit=20000)
    return c.replace(**kw)


def _quick_symbol(vel, h, theta):
    """Semi-discrete symbol of -d/dx (F phi) with the QUICK face value and a
    uniform mass flux F = vel (both upwind branches):
    -|F|/h (1 - cos)^2 / 4 - i F/h (10 sin - sin 2 theta) / 8."""
    c, s, s2 = np.cos(theta), np.sin(theta), np.sin(2 * theta)
    return -abs(vel) / h * (1 - c) ** 2 / 4 - 1j * vel / h * (10 * s - s2) / 8


# --------------------------------------------------------------------------
# (a) QUICK advection of momentum by the u^{n+1/2} mass flux


@pytest.mark.parametrize("U0,V0", [(0.7, -0.55), (-0.6, 0.45)])
def test_momentum_shear_waves_under_rotating_mean_flow(U0, V0):
    """w = W0 + A sin(2 pi m x) + B sin(2 pi m' y) carried by a uniform
    current (U, V) that Coriolis turns during the step.  The current obeys
        u^{k+1} = u^n + dt f ((v^k + v^n)/2 - v_g),
        v^{k+1} = v^n - dt f ((u^k + u^n)/2 - u_g),
    and each wave's complex amplitude W obeys
        W^{k+1} = W^n + dt lam(ubar_k) (W^k + W^n) / 2,  ubar_k = (u^k + u^n)/2,
    lam the QUICK symbol of the advecting component.  The test rules out:
    advecting by u^k (or u^n) instead of u^{n+1/2} -- the current changes
    between sub-iterations, so ubar_k differs from u^k by O(f dt); advecting
    w^k instead of (w^k + w^n)/2, or dropping the 1/2; a wrong upwind branch
    (the signs of U, V and their rotation cover both); and the x / y face
    indexing (the two waves have different wavenumbers)."""
    n, nz, mx, my, steps, K = 32, 4, 3, 2, 20, 3
    h = 1.0 / n
    f, W0, A, B = 4.0, 0.2, 0.3, -0.25
    dt = 0.3 * h / np.hypot(U0, V0)
    c = _case(n, n, nz, h, physics=("adv", "coriolis"), f_cor=f, ug=0.0, vg=0.0, K=K, dt=dt)
    x = (np.arange(n) + 0.5) * h
    X = np.broadcast_to(x[None, None, :], c.shape)
    Y = np.broadcast_to(x[None, :, None], c.shape)
    w0 = W0 + A * np.sin(2 * np.pi * mx * X) + B * np.sin(2 * np.pi * my * Y)
    o = Oracle(c, {"u": np.full(c.shape, U0), "v": np.full(c.shape, V0), "w": w0})
    o.step(steps)

    tx, ty = 2 * np.pi * mx / n, 2 * np.pi * my / n
    u, v = U0, V0
    ax, ay = complex(A), complex(B)
    for _ in range(steps):
        un, vn, axn, ayn = u, v, ax, ay
        uk, vk, axk, ayk = un, vn, axn, ayn
        for _k in range(K):
            ub, vb = 0.5 * (uk + un), 0.5 * (vk + vn)
            ax_new = axn + dt * _quick_symbol(ub, h, tx) * 0.5 * (axk + axn)
            ay_new = ayn + dt * _quick_symbol(vb, h, ty) * 0.5 * (ayk + ayn)
            uk, vk = un + dt * f * vb, vn - dt * f * ub
            axk, ayk = ax_new, ay_new
        u, v, ax, ay = uk, vk, axk, ayk
    i = np.arange(n)
    wx = np.imag(ax * np.exp(1j * tx * (i + 0.5)))
    wy = np.imag(ay * np.exp(1j * ty * (i + 0.5)))
    expect_w = W0 + wx[None, None, :] + wy[None, :, None]
    assert np.max(np.abs(o.get("u") - u)) < 1e-13
    assert np.max(np.abs(o.get("v") - v)) < 1e-13
    assert np.max(np.abs(o.get("w") - expect_w)) < 1e-12
    # the current turned by well over a radian and the waves moved and decayed
    assert abs(np.angle(complex(u, v)) - np.angle(complex(U0, V0))) > 0.5
    assert abs(ax) < 0.99 * A or abs(abs(ax) - A) > 1e-4


@pytest.mark.parametrize("W0", [0.6, -0.45])
def test_momentum_vertical_shear_advection(W0):
    """u = A sin(2 pi m z), v = B cos(2 pi m' z) carried through z by a uniform
    w = W0 (periodic): each mode follows G_K(lam dt)^N with lam the QUICK
    symbol in z.  Rules out a wrong z branch or z-face indexing of the
    momentum fluxes and the averaging of the advected quantity in z."""
    n, m1, m2, steps, K = 32, 3, 5, 15, 3
    h = 1.0 / n
    dt = 0.3 * h / abs(W0)
    c = _case(4, 4, n, h, physics=("adv",), K=K, dt=dt)
    z = (np.arange(n) + 0.5) * h
    Z = np.broadcast_to(z[:, None, None], c.shape)
    A, B = 0.4, -0.3
    o = Oracle(c, {"u": A * np.sin(2 * np.pi * m1 * Z), "v": B * np.cos(2 * np.pi * m2 * Z),
                   "w": np.full(c.shape, W0)})
    o.step(steps)

    def gk(zz):
        g = 1.0 + 0.0j
        for _ in range(K):
            g = 1.0 + 0.5 * zz * (g + 1.0)
        return g

    t1, t2 = 2 * np.pi * m1 / n, 2 * np.pi * m2 / n
    G1 = gk(_quick_symbol(W0, h, t1) * dt) ** steps
    G2 = gk(_quick_symbol(W0, h, t2) * dt) ** steps
    k = np.arange(n)
    eu = np.imag(A * G1 * np.exp(1j * t1 * (k + 0.5)))
    ev = np.real(B * G2 * np.exp(1j * t2 * (k + 0.5)))
    assert np.max(np.abs(o.get("u") - eu[:, None, None])) < 1e-12
    assert np.max(np.abs(o.get("v") - ev[:, None, None])) < 1e-12
    assert np.max(np.abs(o.get("w") - W0)) < 1e-13


# --------------------------------------------------------------------------
# (b) pressure gradient and buoyancy: a discrete rest state


def test_discrete_hydrostatic_rest_state():
    """Walls, the reference state of Eqs. 2-4 (rho0 falls by ~10 % over the
    column), a dry stable theta_l(z) and a pressure p' built so that the
    central difference of alpha0 p' equals the buoyancy b node by node (with
    the mirror ghosts of the walls): the predictor's -rho0 G(alpha0 p') and
    +rho0 b k cancel exactly, so the fluid stays at rest through every
    sub-iteration of several steps.  psi(z) is chosen first, b = G psi, and
    theta_l is obtained from b by inverting the dry thermodynamics of Sec. 2.1
    (b = g (alpha - alpha0) / alpha0, alpha = R_d Pi theta_l / p0, Pi =
    (p0 / p00)^(R_d / c_pd)); p' = rho0 psi.  Rules out: a sign error on G or
    on b; G applied to p' instead of alpha0 p'; rho0 dropped from the
    buoyancy or from the pressure term; a wrong ghost rule for p' at the
    walls."""
    nz, dz, K, steps = 48, 20.0, 3, 3
    c = _case(4, 4, nz, dz, walls=True, physics=("buoy",), rho0_const=None, K=K, dt=2.0,
              theta0=300.0, p00=1.0e5)
    probe = Oracle(c)
    rho0, p0 = probe.profiles()
    alpha0 = 1.0 / rho0
    assert rho0[0] / rho0[-1] > 1.08      # the alpha0 / rho0 factors matter here
    H = nz * dz
    z = (np.arange(nz) + 0.5) * dz
    psi = 60.0 * np.cos(np.pi * z / H) + 15.0 * np.sin(2 * np.pi * z / H) + 5.0
    ghost = np.concatenate(([psi[0]], psi, [psi[-1]]))           # mirror ghosts
    b = (ghost[2:] - ghost[:-2]) / (2 * dz)
    Rd, cpd, g, p00 = 287.0, 1004.5, 9.81, 1.0e5
    alpha = alpha0 * (1.0 + b / g)
    theta = alpha * p0 / Rd / (p0 / p00) ** (Rd / cpd)
    pp = rho0 * psi
    sh = c.shape
    o = Oracle(c, {"u": np.zeros(sh), "v": np.zeros(sh), "w": np.zeros(sh),
                   "theta_l": np.broadcast_to(theta[:, None, None], sh), "q_t": np.zeros(sh),
                   "p": np.broadcast_to(pp[:, None, None], sh)})
    o.begin_step()
    b_orc = o.get("b")[:, 0, 0]
    assert np.max(np.abs(b_orc - b)) < 1e-12 * np.max(np.abs(b))   # the thermodynamics gives b back
    assert np.max(np.abs(b)) > 0.05
    for _ in range(K):
        o.scalar_stage()
        o.momentum_stage()
        for name in ("u_hat", "v_hat", "w_hat"):
            assert np.max(np.abs(o.get(name))) < 1e-12
        o.solve_stage()
        o.correct_stage()
    o.end_step()
    o.step(steps - 1)
    scale = c.dt * np.max(np.abs(b))
    for name in ("u", "v", "w"):
        assert np.max(np.abs(o.get(name))) < 1e-12 * scale
    assert np.max(np.abs(o.get("p")[:, 0, 0] - pp)) < 1e-10 * np.max(np.abs(pp))
    assert np.max(np.abs(o.get("theta_l")[:, 0, 0] - theta)) < 1e-12


# --------------------------------------------------------------------------
# (c) Smagorinsky stress with variable nu_t: first-step energy budget


def _abc(c, A=1.0, B=0.8, C=0.6):
    """Arnold-Beltrami-Childress flow on [0, 1)^3 (divergence-free, and every
    component independent of its own coordinate, so the central divergence
    is exactly zero on the grid)."""
    t = 2 * np.pi
    x = (np.arange(c.nx) + 0.5) * c.dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return {"u": A * np.sin(t * Z) + C * np.cos(t * Y), "v": B * np.sin(t * X) + A * np.cos(t * Z),
            "w": C * np.sin(t * Y) + B * np.cos(t * X)}


def _abc_s3_integral(A=1.0, B=0.8, C=0.6, m=128):
    """int over [0,1)^3 of S^3, S = sqrt(2 S_ij S_ij), of the ABC flow (fine
    periodic midpoint rule on the analytic velocity gradients)."""
    t = 2 * np.pi
    x = (np.arange(m) + 0.5) / m
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    J = np.zeros((3, 3) + Z.shape)          # J[c, d] = d u_c / d x_d
    J[0, 1] = -t * C * np.sin(t * Y)
    J[0, 2] = t * A * np.cos(t * Z)
    J[1, 0] = t * B * np.cos(t * X)
    J[1, 2] = -t * A * np.sin(t * Z)
    J[2, 0] = -t * B * np.sin(t * X)
    J[2, 1] = t * C * np.cos(t * Y)
    S = 0.5 * (J + J.transpose(1, 0, 2, 3, 4))
    s_norm = np.sqrt(2.0 * np.sum(S * S, axis=(0, 1)))
    return float(np.mean(s_norm ** 3))


def _energy(o, c):
    return 0.5 * sum(float(np.sum(o.get(k) ** 2)) for k in ("u", "v", "w")) * c.dx * c.dy * c.dz


def _dissipation_rate(n, dt, cs=0.17):
    h = 1.0 / n
    c = _case(n, n, n, h, physics=("sgs",), cs=cs, K=3, dt=dt, tol=1e-13)
    o = Oracle(c, _abc(c))
    e0 = _energy(o, c)
    o.step(1)
    return (_energy(o, c) - e0) / dt


def test_smagorinsky_energy_budget_first_step():
    """With advection off and a discretely divergence-free ABC flow, the first
    step changes the kinetic energy by -dt eps_h + O(dt^2), and eps_h is the
    Smagorinsky dissipation int rho0 nu_t 2 S_ij S_ij dV = (c_s Delta)^2 int S^3
    dV up to O(Delta^2).  (The pressure does no work at first order: G and the
    central D are negative adjoints and D u^n = 0.)  Checked: (1) the budget
    residual is O(dt^2) -- the rate found with dt and dt/2 differs by twice
    what dt/2 and dt/4 give; (2) the dt -> 0 rate, by Richardson
    extrapolation, equals -(c_s h)^2 int S^3 within 1.5 % at 32^3 and its
    error falls at least 3x from 16^3 to 32^3.  Rules out: the tangential
    stress term with the derivative transposed (d_d u_c twice), a missing
    cross term, the factor 2 in S = sqrt(2 S_ij S_ij), a stress of the wrong
    sign and a dropped 1/2 in u^{n+1/2}."""
    cs = 0.17
    s3 = _abc_s3_integral()
    errs = {}
    for n in (16, 32):
        h = 1.0 / n
        eps = (cs * h) ** 2 * s3
        dt = 0.02
        r1, r2, r4 = (_dissipation_rate(n, dt / q, cs) for q in (1, 2, 4))
        assert r1 < 0 and r2 < 0 and r4 < 0
        # first-order consistency in dt: successive differences halve
        d12, d24 = r1 - r2, r2 - r4
        assert abs(d12 / d24 - 2.0) < 0.05
        rate0 = 2 * r4 - r2
        errs[n] = abs(rate0 / -eps - 1.0)
    assert errs[32] < 0.015
    assert errs[16] / errs[32] > 3.0


def _general_flow(sp, x, y, z):
    """A smooth periodic flow on [0, 1)^3 whose components also vary along
    their own coordinates (so the two nodal cross derivatives on either side
    of a face differ) and whose strain never vanishes: S^2 stays above 4 % of
    its maximum, so nu_t is smooth."""
    t = 2 * sp.pi
    return [sp.sin(t * z) + 0.3 * sp.cos(t * y) + 0.3 * sp.sin(t * (x + y)),
            0.5 * sp.sin(t * x) + sp.cos(t * z) + 0.25 * sp.cos(t * (y + z)),
            0.3 * sp.sin(t * y) + 0.5 * sp.cos(t * x) + 0.2 * sp.sin(t * (z + x))]


def _sgs_force_exact(n, cs):
    """Velocity of the general flow at the nodes of an n^3 grid and its exact
    continuum Smagorinsky force d_d (nu_t (d_d u_c + d_c u_d)), nu_t =
    (c_s Delta)^2 S, Delta = 1/n, differentiated symbolically (sympy)."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    vel = _general_flow(sp, x, y, z)
    X = (x, y, z)
    J = [[sp.diff(vel[c], X[d]) for d in range(3)] for c in range(3)]
    S2 = sum(2 * (sp.Rational(1, 2) * (J[c][d] + J[d][c])) ** 2 for c in range(3) for d in range(3))
    nu = (cs / n) ** 2 * sp.sqrt(S2)
    force = [sum(sp.diff(nu * (J[c][d] + J[d][c]), X[d]) for d in range(3)) for c in range(3)]
    q = (np.arange(n) + 0.5) / n
    Zg, Yg, Xg = np.meshgrid(q, q, q, indexing="ij")
    ev = lambda exprs: [np.broadcast_to(np.asarray(a, dtype=float), Zg.shape).copy()
                        for a in sp.lambdify((x, y, z), exprs, "numpy")(Xg, Yg, Zg)]
    return ev(vel), ev(force)


def test_smagorinsky_force_converges_pointwise():
    """The discrete stress divergence with variable nu_t, node by node, against
    the exact continuum force of a smooth flow (`_general_flow`).  The force
    is read from the first momentum predictor of a step, (u^ - u^n) / dt,
    with advection off and p' = 0.  The largest nodal error, relative to the
    largest force, must fall at second order (at least 3.3x per halving of
    the spacing, 16^3 -> 32^3 -> 64^3).  Rules out first-order slips that an
    integral budget cannot see: the face viscosity or the tangential
    derivative taken from one side of the face, an off-by-one face index, and
    a wrong spacing in a cross term."""
    cs = 0.17
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        c = _case(n, n, n, h, physics=("sgs",), cs=cs, K=1, dt=1e-3)
        vel, exact = _sgs_force_exact(n, cs)
        o = Oracle(c, dict(zip(("u", "v", "w"), vel)))
        o.begin_step()
        o.scalar_stage()
        o.momentum_stage()
        scale = max(np.max(np.abs(e)) for e in exact)
        err = 0.0
        for name, src, ex in zip(("u_hat", "v_hat", "w_hat"), ("u_n", "v_n", "w_n"), exact):
            got = (o.get(name) - o.get(src)) / c.dt
            err = max(err, float(np.max(np.abs(got - ex))) / scale)
        errs.append(err)
    assert errs[1] < 0.02
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3
