"""The decomposed LES step on CPU ranks (gloo, world size 2): the schedule of
paper_2301_04698_gb300.decomp.decomposed_step -- the order of the stages and
of the halo exchanges, with halos two nodes deep -- driven over FP64 oracles
that each hold one widened sub-domain, exchanging through TorchExchange.

The stencil stages evaluate the same arithmetic at every node, so with the
halos right the owned nodes must equal, bit for bit, the single-domain
oracle's: after the step's thermodynamics (every node of the widened domain,
halos included) and after the first scalar and momentum predictors.  The
solve differs only in the order of its sums (its own CG here, with the
one-reduction update of the device solve and one all-reduce per iteration),
so after whole steps the fields agree to the solver tolerance.  The moist
capped boundary layer with every physics term on, plus seeded velocity noise
so that advection and the Smagorinsky stress act in all three directions.
Runs without a GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2301_04698_gb300 import decomp, inputs  # noqa: E402

H = decomp.HALO
NX, NY, NZ = 16, 12, 24
STEPS = 2


def _case():
    return inputs.cbl(nx=NX, ny=NY, nz=NZ, dx=35.0, dz=40.0, precision=64, tol=1e-12, maxit=4000)


def _state(case):
    st = inputs.initial_state(case)
    for s, k in enumerate(("u", "v", "w")):
        st[k] = st[k] + inputs.uniform(5, 40 + s, case.n, -0.5, 0.5).reshape(case.shape)
    return st


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _lc(vp, h, walls):
    """compact Laplacian of a block with a one-node x-y halo, on its interior"""
    hx, hy, hz = h
    c = vp[:, 1:-1, 1:-1]
    zp = np.concatenate([c[1:], c[-1:] if walls else c[:1]], axis=0)
    zm = np.concatenate([c[:1] if walls else c[-1:], c[:-1]], axis=0)
    return ((vp[:, 1:-1, 2:] - 2 * c + vp[:, 1:-1, :-2]) / hx ** 2 +
            (vp[:, 2:, 1:-1] - 2 * c + vp[:, :-2, 1:-1]) / hy ** 2 + (zp - 2 * c + zm) / hz ** 2)


class _OracleRank:
    """One rank: an oracle on the widened sub-domain, halos through gloo."""

    def __init__(self, case, px, py, rank):
        from oracle import Oracle
        self.case = case
        self.rx, self.ry, self.x0, self.y0, self.nx, self.ny = decomp.partition(case.nx, case.ny, px, py, rank)
        self.ex = decomp.TorchExchange(px, py, rank)
        self.o = Oracle(case.replace(nx=self.nx + 2 * H, ny=self.ny + 2 * H))
        self.o.dt = case.dt
        iy, ix = decomp.widened_window(case.nx, case.ny, px, py, rank)
        for k, v in _state(case).items():
            self.o.set(k, v[:, iy][:, :, ix])

    def owned(self, name):
        return self.o.get(name)[:, H:H + self.ny, H:H + self.nx]

    def _swap(self, send):
        recv = [None if t is None else torch.empty_like(t) for t in send]
        self.ex.exchange(send, recv)
        return recv

    def exchange(self, names):
        a = [self.o.view(n) for n in names]
        nx, ny = self.nx, self.ny
        W, E, S, N = decomp.WEST, decomp.EAST, decomp.SOUTH, decomp.NORTH
        send = [None] * 4
        send[W] = torch.from_numpy(np.stack([v[:, H:H + ny, H:2 * H] for v in a]))
        send[E] = torch.from_numpy(np.stack([v[:, H:H + ny, nx:nx + H] for v in a]))
        r = self._swap(send)
        for f, v in enumerate(a):
            v[:, H:H + ny, 0:H] = r[W][f].numpy()
            v[:, H:H + ny, nx + H:nx + 2 * H] = r[E][f].numpy()
        send = [None] * 4
        send[S] = torch.from_numpy(np.stack([v[:, H:2 * H, :] for v in a]))
        send[N] = torch.from_numpy(np.stack([v[:, ny:ny + H, :] for v in a]))
        r = self._swap(send)
        for f, v in enumerate(a):
            v[:, 0:H, :] = r[S][f].numpy()
            v[:, ny + H:ny + 2 * H, :] = r[N][f].numpy()

    def stage(self, name):
        {"begin": self.o.begin_step, "scalar": self.o.scalar_stage, "momentum": self.o.momentum_stage,
         "correct": self.o.correct_stage, "end": self.o.end_step}[name]()

    def _pad1(self, v):
        """v with a one-node halo from the neighbours (the solver's exchange)"""
        W, E, S, N = decomp.WEST, decomp.EAST, decomp.SOUTH, decomp.NORTH
        send = [torch.from_numpy(np.ascontiguousarray(f)) for f in
                (v[:, :, 0], v[:, :, -1], v[:, 0, :], v[:, -1, :])]
        r = self._swap(send)
        vp = np.zeros((v.shape[0], v.shape[1] + 2, v.shape[2] + 2))
        vp[:, 1:-1, 1:-1] = v
        vp[:, 1:-1, 0], vp[:, 1:-1, -1] = r[W].numpy(), r[E].numpy()
        vp[:, 0, 1:-1], vp[:, -1, 1:-1] = r[S].numpy(), r[N].numpy()
        return vp

    def solve(self):
        """the right side again (u^ halos fresh), then CG over the ranks"""
        c = self.case
        self.o.poisson_rhs()
        b = self.owned("rhs")
        ar = lambda vals: self.ex.allreduce(np.asarray(vals, dtype=np.float64))
        ntot = c.nx * c.ny * c.nz
        b = b - ar([b.sum()])[0] / ntot
        bn = np.sqrt(ar([(b * b).sum()])[0])
        x = np.zeros_like(b)
        r, p = b.copy(), b.copy()
        rr = ar([(r * r).sum()])[0]
        it = 0
        while np.sqrt(rr) / bn > c.tol and it < c.maxit:
            q = _lc(self._pad1(p), (c.dx, c.dy, c.dz), c.walls)
            pq, rr0, rq, qq = ar([(p * q).sum(), (r * r).sum(), (r * q).sum(), (q * q).sum()])
            alpha = rr0 / pq
            rr = max(rr0 - 2 * alpha * rq + alpha * alpha * qq, 0.0)
            beta = rr / rr0
            x, r = x + alpha * p, r - alpha * q
            p = r + beta * p
            it += 1
        x = x - ar([x.sum()])[0] / ntot
        psi = self.o.view("psi")
        psi[...] = 0.0
        psi[:, H:H + self.ny, H:H + self.nx] = x
        return {"solves": 1, "iters_total": it, "iters_max": it, "not_converged": int(np.sqrt(rr) / bn > c.tol),
                "res_max": float(np.sqrt(rr) / bn)}


class _OracleWhole:
    """The undivided domain through the same schedule (exchanges are no-ops)."""

    def __init__(self, case):
        from oracle import Oracle
        self.o = Oracle(case, _state(case))
        self.o.dt = case.dt

    def exchange(self, names):
        pass

    def stage(self, name):
        _OracleRank.stage(self, name)

    def solve(self):
        st, it, res = self.o.solve_stage()
        return {"solves": 1, "iters_total": it, "iters_max": it, "not_converged": int(st != 0), "res_max": res}


SNAP = {("begin", 0): ("b", "T", "q_l", "s_rad", "u_n", "theta_l_half"),
        ("momentum", 0): ("theta_l", "q_t", "u_hat", "v_hat", "w_hat")}
FINAL = ("u", "v", "w", "p", "theta_l", "q_t")


def _worker(rank, world, port, px, py, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = _case()
        sd = _OracleRank(case, px, py, rank)
        snaps = {}

        def after(stage, k):
            if (stage, k) in SNAP and (stage, k) not in snaps:
                whole = stage == "begin"      # fresh on the whole widened domain
                snaps[(stage, k)] = {n: (sd.o.get(n) if whole else sd.owned(n)) for n in SNAP[(stage, k)]}

        tot = decomp.decomposed_step(sd, case.K, STEPS, after)
        q.put((rank, sd.x0, sd.y0, snaps, {n: sd.owned(n) for n in FINAL}, tot))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2)])
def test_decomposed_step_on_two_gloo_ranks(px, py):
    case = _case()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, px, py, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0

    ref = _OracleWhole(case)
    snaps = {}

    def after(stage, k):
        if (stage, k) in SNAP and (stage, k) not in snaps:
            snaps[(stage, k)] = {n: ref.o.get(n) for n in SNAP[(stage, k)]}

    tot = decomp.decomposed_step(ref, case.K, STEPS, after)
    final = {n: ref.o.get(n) for n in FINAL}
    for rank, x0, y0, rsnaps, rfinal, rtot in res:
        nyl, nxl = rfinal["u"].shape[1:]
        iy, ix = decomp.widened_window(NX, NY, px, py, rank)
        for n in SNAP[("begin", 0)]:              # halos included
            assert np.array_equal(rsnaps[("begin", 0)][n], snaps[("begin", 0)][n][:, iy][:, :, ix]), n
        for n in SNAP[("momentum", 0)]:
            assert np.array_equal(rsnaps[("momentum", 0)][n],
                                  snaps[("momentum", 0)][n][:, y0:y0 + nyl, x0:x0 + nxl]), n
        for n in FINAL:
            g = final[n][:, y0:y0 + nyl, x0:x0 + nxl]
            scale = np.abs(final[n]).max() + 1e-30
            assert np.abs(rfinal[n] - g).max() <= 1e-9 * scale, (n, np.abs(rfinal[n] - g).max() / scale)
        assert abs(rtot["iters_total"] - tot["iters_total"]) <= 2 * case.K * STEPS
        assert rtot["not_converged"] == 0
    assert res[0][5]["iters_total"] == res[1][5]["iters_total"]   # the ranks agree


def test_widened_window_wraps():
    iy, ix = decomp.widened_window(10, 8, 2, 2, 3)     # rank 3: rx = 1, ry = 1
    assert list(ix) == [3, 4, 5, 6, 7, 8, 9, 0, 1]
    assert list(iy) == [2, 3, 4, 5, 6, 7, 0, 1]
