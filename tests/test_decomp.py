"""The multi-rank path of the decomposed Poisson solve on CPU ranks (gloo,
world size 2): the partition, the neighbour map and the halo exchange /
all-reduce protocol of paper_2301_04698_gb300.decomp, which the device solve
(les_dd_poisson_solve) calls once per CG iteration.

Checked on two x-y layouts (2 x 1 and 1 x 2): after one exchange every halo
strip equals, bit for bit, the neighbouring nodes of the periodic global
field; and a CG written here in numpy that uses only the local part, the
exchange and the all-reduce -- the same steps as the device solve -- gives the
FP64 oracle's single-domain solution (Sec. 2.4, compact operator, walls in z)
to the solver tolerance.  Runs without a GPU.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2301_04698_gb300 import decomp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


NX, NY, NZ, H = 12, 10, 6, (40.0, 35.0, 10.0)


def _global_field(seed):
    from paper_2301_04698_gb300 import inputs
    return inputs.uniform(seed, 0, NX * NY * NZ, -1, 1).reshape(NZ, NY, NX)


def _faces(v):
    """the four face strips of an interior block v (nz, ny, nx): in-face
    index fastest, then z"""
    return [np.ascontiguousarray(v[:, :, 0]), np.ascontiguousarray(v[:, :, -1]),
            np.ascontiguousarray(v[:, 0, :]), np.ascontiguousarray(v[:, -1, :])]


def _exchange_np(ex, v):
    send = [torch.from_numpy(f.copy()) for f in _faces(v)]
    recv = [torch.empty_like(t) for t in send]
    ex.exchange(send, recv)
    return [r.numpy() for r in recv]


def _lc(vp, walls=True):
    """compact Laplacian of the padded block (halo 1 in x, y) on its interior"""
    hx, hy, hz = H
    c = vp[:, 1:-1, 1:-1]
    zp = np.concatenate([c[1:], c[-1:] if walls else c[:1]], axis=0)
    zm = np.concatenate([c[:1] if walls else c[-1:], c[:-1]], axis=0)
    return ((vp[:, 1:-1, 2:] - 2 * c + vp[:, 1:-1, :-2]) / hx ** 2 +
            (vp[:, 2:, 1:-1] - 2 * c + vp[:, :-2, 1:-1]) / hy ** 2 + (zp - 2 * c + zm) / hz ** 2)


def _pad(ex, v):
    r = _exchange_np(ex, v)
    vp = np.zeros((v.shape[0], v.shape[1] + 2, v.shape[2] + 2))
    vp[:, 1:-1, 1:-1] = v
    vp[:, 1:-1, 0], vp[:, 1:-1, -1], vp[:, 0, 1:-1], vp[:, -1, 1:-1] = r[0], r[1], r[2], r[3]
    return vp


def _dd_cg(ex, b, tol, maxit):
    """CG on this rank's part with the one-reduction update of the device solve"""
    ar = lambda vals: ex.allreduce(np.asarray(vals, dtype=np.float64))
    ntot = NX * NY * NZ
    b = b - ar([b.sum()])[0] / ntot
    bn = np.sqrt(ar([(b * b).sum()])[0])
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = ar([(r * r).sum()])[0]
    it = 0
    while np.sqrt(rr) / bn > tol and it < maxit:
        q = _lc(_pad(ex, p))
        pq, rr0, rq, qq = ar([(p * q).sum(), (r * r).sum(), (r * q).sum(), (q * q).sum()])
        alpha = rr0 / pq
        rr = max(rr0 - 2 * alpha * rq + alpha * alpha * qq, 0.0)
        beta = rr / rr0
        x = x + alpha * p
        r = r - alpha * q
        p = r + beta * p
        it += 1
    x = x - ar([x.sum()])[0] / ntot
    return x, it


def _worker(rank, world, port, px, py, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rx, ry, x0, y0, nxl, nyl = decomp.partition(NX, NY, px, py, rank)
        ex = decomp.TorchExchange(px, py, rank)
        g = _global_field(3)
        v = g[:, y0:y0 + nyl, x0:x0 + nxl]
        r = _exchange_np(ex, v)
        # the halo strips are the periodic neighbours of the block
        want = [g[:, y0:y0 + nyl, (x0 - 1) % NX], g[:, y0:y0 + nyl, (x0 + nxl) % NX],
                g[:, (y0 - 1) % NY, x0:x0 + nxl], g[:, (y0 + nyl) % NY, x0:x0 + nxl]]
        halo_ok = all(np.array_equal(a, b) for a, b in zip(r, want))
        # decomposed CG on a right side of the operator's range
        b = _global_field(7)
        x, it = _dd_cg(ex, b[:, y0:y0 + nyl, x0:x0 + nxl], 1e-12, 2000)
        q.put((rank, halo_ok, x0, y0, x, it))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2)])
def test_decomposed_solve_on_two_gloo_ranks(px, py):
    from oracle import Oracle
    from paper_2301_04698_gb300 import inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, px, py, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = sorted((q.get(timeout=10) for _ in range(2)), key=lambda t: t[0])
    assert all(r[1] for r in res), "halo strips differ from the periodic neighbours"
    assert res[0][5] == res[1][5]                    # the ranks agree on the iteration count
    xg = np.zeros((NZ, NY, NX))
    for rank, _, x0, y0, x, _ in res:
        xg[:, y0:y0 + x.shape[1], x0:x0 + x.shape[2]] = x
    case = inputs.Case(name="dd", nx=NX, ny=NY, nz=NZ, dx=H[0], dy=H[1], dz=H[2], walls=True, precision=64,
                       init="zero", physics=())
    ref, st, it, res_ = Oracle(case).poisson(_global_field(7), tol=1e-12)
    assert np.linalg.norm(xg - ref) / np.linalg.norm(ref) < 1e-9
    assert abs(res[0][5] - it) <= 2


def test_neighbours_wrap_and_pair_up():
    """Every rank's east neighbour has it as its west neighbour, and so on;
    with one partition along an axis a rank is its own neighbour there."""
    for px, py in ((1, 1), (2, 1), (3, 2), (4, 4)):
        for r in range(px * py):
            nb = decomp.neighbours(px, py, r)
            assert decomp.neighbours(px, py, nb[decomp.EAST])[decomp.WEST] == r
            assert decomp.neighbours(px, py, nb[decomp.NORTH])[decomp.SOUTH] == r
            if px == 1:
                assert nb[decomp.EAST] == nb[decomp.WEST] == r
    with pytest.raises(ValueError):
        decomp.partition(10, 8, 3, 1, 0)
