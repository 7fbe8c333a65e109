"""The paper's validation workloads (Sec. 3): the density current and the
rising bubble, as seeded-free synthetic inputs, and the FP64 oracle on them.

The paper shows these cases only as figures, so the oracle is pinned here by
what the mathematics fixes for them: the fields stay independent of y (the
cases are two-dimensional), v stays zero, the solution stays mirror-symmetric
about the bubble's vertical axis (every operator of the scheme is
reflection-equivariant), the integral of rho0 theta is conserved (flux form,
no flux through the walls, no sources), and the bubble moves the way its
buoyancy points."""
import numpy as np
import pytest

from paper_2301_04698_gb300 import inputs


@pytest.mark.parametrize("builder,amp,radii", [(inputs.density_current, -15.0, (4000.0, 2000.0)),
                                               (inputs.rising_bubble, 2.0, (2000.0, 2000.0))])
def test_bubble_initial_fields(builder, amp, radii):
    """Amplitude, radii, domain and the cosine-squared bell as stated (Sec. 3)."""
    c = builder(400.0)
    a = c.init_args
    assert (a["amp"], (a["xr"], a["zr"])) == (amp, radii)
    assert c.walls and c.nu_const in (10.0, 1.0) and "const_nu" in c.physics and "sgs" not in c.physics
    width, height = (51200.0, 6400.0) if amp < 0 else (20000.0, 10000.0)
    assert (c.nx * c.dx, c.nz * c.dz) == (width, height)
    st = inputs.initial_state(c)
    tp = st["theta_l"] - 300.0
    assert float(np.abs(tp - tp[:, :1, :]).max()) == 0.0          # uniform in y
    assert float(np.abs(tp - tp[:, :, ::-1]).max()) == 0.0        # mirror-symmetric about xc
    x = (np.arange(c.nx) + 0.5) * c.dx
    z = (np.arange(c.nz) + 0.5) * c.dz
    L = np.sqrt(((x[None, :] - a["xc"]) / a["xr"]) ** 2 + ((z[:, None] - a["zc"]) / a["zr"]) ** 2)
    assert np.all(tp[:, 0, :][L > 1.0] == 0.0)
    inside = L <= 1.0
    # cos^2(pi L / 2) = (1 + cos(pi L)) / 2: half the amplitude at half the radius
    np.testing.assert_allclose(tp[:, 0, :][inside], 0.5 * amp * (1.0 + np.cos(np.pi * L[inside])), rtol=0, atol=1e-12)
    assert abs(float(np.abs(tp).max())) <= abs(amp) and abs(float(np.abs(tp).max())) > 0.9 * abs(amp)
    for k in ("u", "v", "w", "q_t"):
        assert float(np.abs(st[k]).max()) == 0.0


@pytest.mark.parametrize("builder,dx,sign", [(inputs.density_current, 800.0, -1.0),
                                             (inputs.rising_bubble, 400.0, 1.0)])
def test_oracle_bubble_invariants(builder, dx, sign):
    """20 FP64 oracle steps: y-independence and v = 0 exactly, mirror symmetry
    to rounding, conservation of the rho0-weighted theta, and the bubble's
    vertical velocity along its buoyancy."""
    from oracle import Oracle
    c = builder(dx)
    o = Oracle(c, inputs.initial_state(c))
    rho0 = o.profiles()[0]
    m0 = float((rho0[:, None, None] * o.get("theta_l")).sum())
    o.step(20)
    th, u, v, w = (o.get(k) for k in ("theta_l", "u", "v", "w"))
    tp = th - 300.0
    for f in (th, u, w):
        assert float(np.abs(f - f[:, :1, :]).max()) == 0.0
    assert float(np.abs(v).max()) == 0.0
    assert float(np.abs(tp - tp[:, :, ::-1]).max()) <= 1e-11 * float(np.abs(tp).max())
    assert float(np.abs(u + u[:, :, ::-1]).max()) <= 1e-11 * float(np.abs(u).max())
    assert float(np.abs(w - w[:, :, ::-1]).max()) <= 1e-11 * float(np.abs(w).max())
    m1 = float((rho0[:, None, None] * th).sum())
    assert abs(m1 - m0) <= 1e-13 * abs(m0)
    # at the bubble's centre the flow follows its buoyancy
    a = c.init_args
    ic = int(a["xc"] / c.dx) - 1  # the node left of the axis (nx even: the axis is a face)
    kc = int(a["zc"] / c.dz)
    assert sign * w[kc, 0, ic] > 0.5
