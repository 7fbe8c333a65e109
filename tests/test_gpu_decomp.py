"""The decomposed Poisson solve (les_dd_poisson_solve) on one GPU: the
sub-domains of a px x py partition, each solved by its own host thread on its
own stream, exchange their halos through the same callback interface that
NCCL sends and receives sit behind between GPUs (here device copies,
decomp.LocalExchange), and must reach the single-domain solve
(les_poisson_solve) of the whole grid: the same iterates up to the order of
the sums, so the same iteration count within one and the same solution to
the tolerance.  The kernels of different sub-domains never wait for each
other on the device; the threads meet on the host."""
import threading

import numpy as np
import pytest

from paper_2301_04698_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_04698_gb300 import build, decomp, les
    build.build()
    les.load_library()
    return les, decomp


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,walls,px,py,shape", [
    (64, True, 2, 2, (48, 40, 12)), (64, False, 2, 1, (32, 24, 10)), (32, True, 2, 2, (64, 48, 16)),
    (64, True, 4, 1, (64, 16, 8))])
def test_decomposed_solve_matches_single_domain(mods, precision, walls, px, py, shape):
    les, decomp = mods
    nx, ny, nz = shape
    case = inputs.Case(name="dd", nx=nx, ny=ny, nz=nz, dx=40.0, dy=35.0, dz=10.0, walls=walls, precision=precision,
                       init="zero", physics=(), rho0_const=1.0)
    tol = 1e-10 if precision == 64 else 1e-6
    dt = torch.float64 if precision == 64 else torch.float32
    sim = les.Simulation(case)
    xt = torch.from_numpy(inputs.uniform(17, 0, case.n, -1, 1).reshape(case.shape)).to("cuda", dt)
    b = sim.apply_poisson(xt, "compact")
    x_ref = torch.zeros_like(b)
    rc, it_ref, res_ref = sim.poisson_solve(b, x_ref, tol, 5000)
    torch.cuda.synchronize()
    ex = decomp.LocalExchange(px, py)
    subs = [decomp.Subdomain(case, px, py, r) for r in range(px * py)]
    out = [None] * len(subs)
    errors = []

    def run(r):
        try:
            s = subs[r]
            torch.cuda.set_device(0)
            rhs = s.local(b).contiguous()
            x = torch.zeros_like(rhs)
            rcode, it, rel = s.solve(rhs, x, tol, 5000,
                                     lambda send, recv, stream: ex.exchange(r, send, recv, stream),
                                     lambda vals: ex.allreduce(r, vals))
            out[r] = (rcode, it, rel, x.cpu().double().numpy())
        except Exception as e:  # surfaced below
            errors.append(e)
            ex.barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(len(subs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(300)
    assert not errors, errors[0]
    xg = np.zeros(case.shape)
    for r, s in enumerate(subs):
        rcode, it, rel, x = out[r]
        assert rcode == les.LES_OK and rel <= tol
        xg[:, s.y0:s.y0 + s.ny, s.x0:s.x0 + s.nx] = x
    its = {o[1] for o in out}
    assert len(its) == 1                         # every rank ran the same iterations
    it = its.pop()
    print(f"{px}x{py} sub-domains: {it} iterations (single domain {it_ref})")
    assert abs(it - it_ref) <= (1 if precision == 64 else 3)
    assert _rel(xg, x_ref.cpu().double().numpy()) < (1e-9 if precision == 64 else 1e-5)
    for s in subs:
        s.close()
    sim.close()


def test_decomposed_solve_rejects_bad_partitions(mods):
    les, decomp = mods
    case = inputs.Case(name="dd", nx=30, ny=24, nz=8, dx=1.0, dy=1.0, dz=1.0, walls=True, precision=64,
                       init="zero", physics=())
    with pytest.raises(Exception):
        decomp.Subdomain(case, 4, 1, 0)          # 4 does not divide 30
    with pytest.raises(Exception):
        decomp.Subdomain(case.replace(op="wide"), 2, 1, 0)


# ---- the decomposed step ------------------------------------------------------

STEPS = 2
SNAP = {("begin", 0): ("b", "T", "q_l", "s_rad", "u_n", "theta_l_half"),
        ("momentum", 0): ("theta_l", "q_t", "u_hat", "v_hat", "w_hat")}
FINAL = ("u", "v", "w", "p", "theta_l", "q_t")


def _cbl_state(case):
    st = inputs.initial_state(case)
    for s, k in enumerate(("u", "v", "w")):
        st[k] = st[k] + inputs.uniform(5, 40 + s, case.n, -0.5, 0.5).reshape(case.shape)
    return st


class _Whole:
    """The undivided domain through the same schedule (no exchanges)."""

    def __init__(self, sim):
        self.sim = sim

    def exchange(self, names):
        pass

    def stage(self, name):
        self.sim.stage(name)

    def solve(self):
        return self.sim.stage("solve")


@pytest.mark.parametrize("precision,px,py,warm", [(64, 2, 2, "zero"), (64, 2, 1, "zero"), (64, 1, 2, "zero"),
                                                  (32, 2, 2, "zero"), (64, 2, 2, "prev")])
def test_decomposed_step_matches_single_domain(mods, precision, px, py, warm):
    """Sub-domains of one GPU, each stepped by its own thread through
    decomp.decomposed_step with the library's halo exchange (two-node halos,
    LocalExchange) and decomposed solve, against the single-domain step on
    the same kernels (the rolling predictors on both): after the step's
    thermodynamics every node of each widened sub-domain, halos included,
    and after the first predictors every owned node equal bit for bit; after
    two steps the fields equal to the solver tolerance.  With the previous
    solution as first guess ("prev") both sides start each solve from their
    own previous psi."""
    les, decomp = mods
    case = inputs.cbl(nx=32, ny=24, nz=24, dx=35.0, dz=40.0, precision=precision,
                      tol=1e-10 if precision == 64 else 1e-6, warm=warm)
    state = _cbl_state(case)
    sim = les.Simulation(case)
    sim.set_tuning(stencil_path=1)
    sim.set_state(state)
    snaps = {}

    def after(stage, k):
        if (stage, k) in SNAP and (stage, k) not in snaps:
            snaps[(stage, k)] = {n: sim.get(n) for n in SNAP[(stage, k)]}

    tot = decomp.decomposed_step(_Whole(sim), case.K, STEPS, after)
    final = {n: sim.get(n) for n in FINAL}
    sim.close()

    ex = decomp.LocalExchange(px, py)
    nr = px * py
    subs = []
    for r in range(nr):
        sd = decomp.DecomposedSimulation(case, px, py, r, lambda s, rv, st, r=r: ex.exchange(r, s, rv, st),
                                         lambda v, r=r: ex.allreduce(r, v))
        sd.sim.set_tuning(stencil_path=1)
        sd.set_global_state(state)
        subs.append(sd)
    out = [None] * nr
    errors = []

    def run(r):
        try:
            torch.cuda.set_device(0)
            sd = subs[r]
            mine = {}

            def grab(stage, k):
                if (stage, k) in SNAP and (stage, k) not in mine:
                    mine[(stage, k)] = {n: (sd.sim.get(n) if stage == "begin" else sd.owned(n))
                                        for n in SNAP[(stage, k)]}

            t = sd.step(STEPS, grab)
            out[r] = (mine, {n: sd.owned(n) for n in FINAL}, t)
        except Exception as e:  # surfaced below
            errors.append(e)
            ex.barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(nr)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(600)
    assert not errors, errors[0]
    rtol = 1e-8 if precision == 64 else 2e-4
    for r, sd in enumerate(subs):
        mine, fin, t = out[r]
        iy, ix = sd.window
        for n in SNAP[("begin", 0)]:
            assert np.array_equal(mine[("begin", 0)][n], snaps[("begin", 0)][n][:, iy][:, :, ix]), n
        ys, xs = slice(sd.sub.y0, sd.sub.y0 + sd.sub.ny), slice(sd.sub.x0, sd.sub.x0 + sd.sub.nx)
        for n in SNAP[("momentum", 0)]:
            assert np.array_equal(mine[("momentum", 0)][n], snaps[("momentum", 0)][n][:, ys, xs]), n
        for n in FINAL:
            g = final[n][:, ys, xs].astype(np.float64)
            scale = np.abs(final[n]).max() + 1e-30
            err = np.abs(fin[n].astype(np.float64) - g).max() / scale
            assert err <= rtol, (n, err)
        assert t["not_converged"] == 0
        print(f"rank {r}: {t['iters_total']} CG iterations over {STEPS} steps (single domain {tot['iters_total']})")
    assert len({out[r][2]["iters_total"] for r in range(nr)}) == 1
    for sd in subs:
        sd.close()


def test_decomposed_step_rejects_a_plain_handle(mods):
    """les_dd_halo_exchange and les_dd_stage_solve refuse a handle that is not
    the widened sub-domain, and the solve stage keeps the stage order."""
    les, decomp = mods
    import ctypes as C
    case = inputs.cbl(nx=32, ny=24, nz=24, dx=35.0, dz=40.0, precision=64)
    ex = decomp.LocalExchange(2, 1)
    sd = decomp.DecomposedSimulation(case, 2, 1, 0, lambda s, rv, st: ex.exchange(0, s, rv, st),
                                     lambda v: ex.allreduce(0, v))
    plain = les.Simulation(case)
    ids = (C.c_int32 * 1)(les.FIELDS["u"])
    assert sd.lib.les_dd_halo_exchange(sd.sub.h, plain.h, sd._opsp, 1, ids) == les.LES_ERR_INVALID_ARG
    st = les.LesStepStats()
    assert sd.lib.les_dd_stage_solve(sd.sub.h, sd.sim.h, sd._opsp, C.byref(st)) == les.LES_ERR_STATE
    two = (C.c_int32 * 2)(les.FIELDS["u"], les.FIELDS["u"])
    assert sd.lib.les_dd_halo_exchange(sd.sub.h, sd.sim.h, sd._opsp, 2, two) == les.LES_ERR_INVALID_ARG
    plain.close()
    sd.close()
