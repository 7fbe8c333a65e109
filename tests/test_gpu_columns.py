"""The column-march stencil kernels (z windows in registers), through the C
ABI, against the FP64 oracle stage by stage.

The correction and the right side run by default on grids whose nx is a
multiple of 32 lanes x (16 bytes / element size), the predictors on grids
whose nx is a multiple of 64 (two nodes per lane), both with ny a multiple of
8; the FP64 instantiation is held to the same bars as the other stencil paths,
with every physics term on and with the dry set (advection and Smagorinsky
only), which the predictors compile as a separate specialisation.  Edge cases: one tile across x (the edge lanes wrap onto the
same tile), one tile across y (the rows j -+ 2 wrap inside the tile), the
fewest planes (nz = 2 with walls) and both boundary conditions.  The FP32
instantiation is compared with the rolling kernels on the same inputs.
"""
import numpy as np
import pytest

from paper_2301_04698_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def les_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_04698_gb300 import build, les
    build.build()
    les.load_library()
    return les


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def demean(a):
    return a - a.mean()


def _state(case, seed=8):
    st = inputs.initial_state(case)
    n, s = case.n, case.shape
    for i, k in enumerate(("u", "v", "w")):
        st[k] = st[k] + inputs.uniform(seed, i, n, -1, 1).reshape(s)
    st["p"] = 10.0 * inputs.uniform(seed, 5, n, -1, 1).reshape(s)
    return st


def _moist(nx, ny, nz, walls, advection="quick", precision=64):
    c = inputs.cbl(nx, ny, nz, dz=70.0, precision=precision, tol=1e-13 if precision == 64 else 1e-6,
                   maxit=5000, sat_tol=1e-10 if precision == 64 else 1e-4, advection=advection)
    if not walls:
        c = c.replace(walls=False, physics=("adv", "sgs", "fb", "moist", "buoy", "coriolis"))
    return c


@pytest.mark.parametrize("shape,walls,advection", [
    ((64, 16, 12), True, "quick"), ((128, 8, 10), False, "quick"), ((64, 8, 2), True, "quick"),
    ((64, 24, 9), False, "weno3"), ((192, 8, 6), True, "weno3")])
def test_column_stages_fp64(les_mod, shape, walls, advection):
    """Stage-by-stage FP64 parity of the default path: every stencil stage as
    a column march."""
    from oracle import Oracle
    case = _moist(*shape, walls, advection)
    st = _state(case)
    sim = les_mod.Simulation(case)
    sim.set_state(st)
    ref = Oracle(case, st)
    assert sim.tuning()["stencil_path"] == 0
    sim.stage("begin")
    ref.begin_step()
    for k in range(case.K):
        sim.stage("scalar")
        ref.scalar_stage()
        for f in ("theta_l", "q_t"):
            assert rel(sim.get(f), ref.get(f)) < 1e-13, (k, f)
        sim.stage("momentum")
        ref.momentum_stage()
        for f in ("u_hat", "v_hat", "w_hat"):
            assert rel(sim.get(f), ref.get(f)) < 1e-12, (k, f)
        assert rel(sim.get("rhs"), ref.get("rhs")) < 1e-10, k
        sim.stage("solve")
        ref.solve_stage()
        assert rel(sim.get("psi"), ref.get("psi")) < 1e-9, k
        sim.stage("correct")
        ref.correct_stage()
        for f in ("u", "v", "w"):
            assert rel(sim.get(f), ref.get(f)) < 1e-9, (k, f)
        assert rel(demean(sim.get("p")), demean(ref.get("p"))) < 1e-9, k
    sim.stage("end")
    ref.end_step()


@pytest.mark.parametrize("shape", [(64, 16, 12), (192, 8, 5)])
def test_column_stages_fp64_dry(les_mod, shape):
    """The dry Taylor-Green physics (advection and Smagorinsky only, periodic,
    the predictors' compile-time specialisation) stage by stage against the
    oracle."""
    from oracle import Oracle
    case = inputs.tgv(32, nxyz=shape, precision=64, steps_tol=1e-13)
    st = _state(case)
    st["theta_l"] = st["theta_l"] + inputs.uniform(9, 6, case.n, -1, 1).reshape(case.shape)
    st["q_t"] = 5e-3 + 1e-3 * inputs.uniform(9, 7, case.n, -1, 1).reshape(case.shape)
    sim = les_mod.Simulation(case)
    sim.set_state(st)
    ref = Oracle(case, st)
    sim.stage("begin")
    ref.begin_step()
    assert sim.dt == ref.dt
    for k in range(case.K):
        sim.stage("scalar")
        ref.scalar_stage()
        for f in ("theta_l", "q_t"):
            assert rel(sim.get(f), ref.get(f)) < 1e-13, (k, f)
        sim.stage("momentum")
        ref.momentum_stage()
        for f in ("u_hat", "v_hat", "w_hat"):
            assert rel(sim.get(f), ref.get(f)) < 1e-12, (k, f)
        sim.stage("solve")
        ref.solve_stage()
        sim.stage("correct")
        ref.correct_stage()
        for f in ("u", "v", "w"):
            assert rel(sim.get(f), ref.get(f)) < 1e-9, (k, f)
    sim.stage("end")
    ref.end_step()


@pytest.mark.parametrize("op", ["compact", "wide"])
def test_column_rhs_and_correct_fp64_exact_inputs(les_mod, op):
    """The right side node by node against the oracle's, with the compact
    operator (Appendix A term) and with the consistent operator."""
    from oracle import Oracle
    case = _moist(128, 16, 7, True).replace(op=op)
    st = _state(case, seed=4)
    sim = les_mod.Simulation(case)
    sim.set_state(st)
    ref = Oracle(case, st)
    sim.stage("begin")
    ref.begin_step()
    sim.stage("scalar")
    ref.scalar_stage()
    sim.stage("momentum")
    ref.momentum_stage()
    assert np.max(np.abs(sim.get("rhs") - ref.get("rhs"))) <= 1e-11 * np.max(np.abs(ref.get("rhs")))


@pytest.mark.parametrize("shape,walls", [((128, 16, 24), True), ((256, 8, 10), False), ((128, 8, 2), True),
                                         ((192, 16, 6), False)])
def test_column_fp32_matches_rolling(les_mod, shape, walls):
    """FP32: the column kernels and the rolling kernels (stencil_path 1) on the
    same inputs agree to float rounding, stage by stage, for three steps.  The
    two round differently (the column predictors scale the tendency by
    dt / rho0, the rolling ones divide rho0 phi + dt T by rho0; their x faces
    are summed in other groupings), and nine sub-iterations amplify the
    differences: 5e-6 relative for u^ (about 40 ulps of float), 1e-4 for the
    right side (a difference of nearly equal fluxes) and 1e-5 for the fields."""
    case = _moist(*shape, walls, precision=32).replace(dt=0.5)
    st = _state(case)
    sims = []
    for path in (0, 1):
        s = les_mod.Simulation(case)
        s.set_state(st)
        s.set_tuning(stencil_path=path)
        sims.append(s)
    for step in range(3):
        for stg in ["begin"] + ["scalar", "momentum", "solve", "correct"] * case.K + ["end"]:
            for s in sims:
                s.stage(stg, allow_not_converged=True)
            if stg == "momentum":
                for f in ("u_hat", "v_hat", "w_hat", "rhs"):
                    a, b = sims[0].get(f), sims[1].get(f)
                    assert rel(a, b) < (1e-4 if f == "rhs" else 5e-6), (step, f)
    for f in ("u", "v", "w", "theta_l", "q_t"):
        assert rel(sims[0].get(f), sims[1].get(f)) < 1e-5, f
