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
