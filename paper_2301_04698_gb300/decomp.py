"""Domain decomposition of the Poisson solve: partition, neighbours and the
halo-exchange / all-reduce functions behind les_dd_poisson_solve.

The paper parallelises its LES by cutting the domain into partitions, one per
TPU core, exchanging halos before every stencil pass and reducing the
solver's sums over all partitions (Sec. 2.5; the partitionings of Sec. 4.2).
Here the global nx x ny x nz grid (periodic in x and y) is cut into px x py
sub-domains with whole z columns; rank r owns sub-domain (rx, ry) = (r % px,
r // px).  The library (les_dd_*) runs the CG on the device and calls back,
once per iteration, to exchange the four face strips of the search direction
and to sum four FP64 values over the ranks.  This module only moves data:

* ``TorchExchange`` -- between processes with torch.distributed (NCCL between
  GPUs, gloo for CPU tensors): point-to-point sends and receives posted in a
  fixed order by direction of travel (eastward, westward, northward,
  southward), so that in-order matching pairs them even when a rank's west
  and east neighbours are the same rank;
* ``LocalExchange`` -- between sub-domains held by threads of one process
  (one device or several), by device copies.

The whole step runs decomposed too (``DecomposedSimulation``): each rank keeps
its fields in a handle widened by two halo nodes on each side in x and y and
follows ``decomposed_step``, the order of stages and exchanges, with the
library's halo packing and decomposed solve.  A strip given as None (0 bytes)
is neither sent nor received: the field halos move in two exchanges, the x
strips and then the y strips, which carry the corners.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3
OPPOSITE = {WEST: EAST, EAST: WEST, SOUTH: NORTH, NORTH: SOUTH}
# (face sent, neighbour it goes to, halo it fills on the receiver), in the
# posting order: a strip travelling east is a rank's east face, sent to its
# east neighbour, which receives it into its west halo
TRAVEL = ((EAST, EAST, WEST), (WEST, WEST, EAST), (NORTH, NORTH, SOUTH), (SOUTH, SOUTH, NORTH))


def partition(nx: int, ny: int, px: int, py: int, rank: int):
    """(rx, ry, x0, y0, nxl, nyl) of `rank` in a px x py partition."""
    if nx % px or ny % py:
        raise ValueError("px must divide nx and py must divide ny")
    rx, ry = rank % px, rank // px
    nxl, nyl = nx // px, ny // py
    return rx, ry, rx * nxl, ry * nyl, nxl, nyl


def neighbours(px: int, py: int, rank: int) -> dict:
    """Ranks on the four sides (periodic)."""
    rx, ry = rank % px, rank // px
    return {WEST: ((rx - 1) % px) + px * ry, EAST: ((rx + 1) % px) + px * ry,
            SOUTH: rx + px * ((ry - 1) % py), NORTH: rx + px * ((ry + 1) % py)}


class TorchExchange:
    """Halo exchange and all-reduce over a torch.distributed process group.
    ``exchange(send, recv)`` takes the four face strips of this rank and
    fills the four halo strips (torch tensors on the group's device).  With
    the gloo backend, device strips travel through host copies (gloo moves
    host memory); with NCCL they go device to device."""

    def __init__(self, px: int, py: int, rank: int, group=None):
        self.px, self.py, self.rank, self.group = px, py, rank, group
        self.nb = neighbours(px, py, rank)

    def exchange(self, send, recv, stream=None) -> None:
        """send / recv: the four face strips and halo strips of this rank;
        stream: the CUDA stream that wrote the strips (or None on the CPU)."""
        import torch
        import torch.distributed as dist
        if stream is not None:
            stream.synchronize()
        staged = dist.get_backend(self.group) == "gloo"
        ops = []
        local = []
        back = []
        for face, side, halo in TRAVEL:
            if send[face] is None:              # this axis is not exchanged now
                continue
            dst = self.nb[side]                 # where this rank's strip goes
            src = self.nb[OPPOSITE[side]]       # whose strip fills the halo
            if dst == self.rank and src == self.rank:
                local.append((halo, face))
                continue
            s, r = send[face], recv[halo]
            if staged and s.is_cuda:
                s = s.cpu()
                r = torch.empty(recv[halo].shape, dtype=recv[halo].dtype)
                back.append((recv[halo], r))
            ops.append(dist.P2POp(dist.isend, s, dst, self.group))
            ops.append(dist.P2POp(dist.irecv, r, src, self.group))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        for dev, host in back:
            dev.copy_(host)
        for halo, face in local:                # periodic with itself
            recv[halo].copy_(send[face])
        if stream is not None:
            torch.cuda.synchronize()            # halos in place before the unpack

    def allreduce(self, values: np.ndarray, device="cpu") -> np.ndarray:
        import torch
        import torch.distributed as dist
        t = torch.from_numpy(np.ascontiguousarray(values, dtype=np.float64)).to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()


class LocalExchange:
    """Sub-domains of one process, each solved by its own thread on its own
    stream: at every exchange the threads meet at a barrier once their face
    strips are written, copy their halos from the neighbours' strips, and
    meet again before any strip is overwritten; the all-reduce sums in rank
    order, so every thread gets the same bits."""

    def __init__(self, px: int, py: int):
        self.px, self.py, self.n = px, py, px * py
        self.barrier = threading.Barrier(self.n)
        self.send = [None] * self.n
        self.vals = [None] * self.n

    def exchange(self, rank: int, send, recv, stream) -> None:
        stream.synchronize()                    # this rank's strips are written
        self.send[rank] = send
        self.barrier.wait()
        nb = neighbours(self.px, self.py, rank)
        import torch
        with torch.cuda.stream(stream):
            for face, side, halo in TRAVEL:
                if recv[halo] is None:
                    continue
                src = nb[OPPOSITE[side]]
                recv[halo].copy_(self.send[src][face])
        stream.synchronize()
        self.barrier.wait()                     # every copy of every strip is done

    def allreduce(self, rank: int, values: np.ndarray) -> np.ndarray:
        self.vals[rank] = np.array(values, dtype=np.float64)
        self.barrier.wait()
        total = np.zeros_like(self.vals[rank])
        for r in range(self.n):
            total = total + self.vals[r]
        self.barrier.wait()
        return total


# ---- binding of les_dd_* ------------------------------------------------------

_EXCHANGE = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_size_t),
                        C.c_void_p)
_ALLREDUCE = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_int32)


class _Ops(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("exchange", _EXCHANGE), ("allreduce", _ALLREDUCE)]


class _DevBuf:
    """A raw device buffer as a torch tensor (CUDA array interface)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "strides": None,
                                         "version": 3}


def _view(ptr: int, nbytes: int):
    import torch
    return torch.as_tensor(_DevBuf(ptr, nbytes), device="cuda")


class Subdomain:
    """One sub-domain of a px x py partition (les_dd_*) for the compact
    Poisson operator of a case (inputs.Case)."""

    def __init__(self, case, px: int, py: int, rank: int, stream=None):
        import torch

        from . import les
        self.lib = les.load_library()
        self.case = case
        self.px, self.py, self.rank = px, py, rank
        self.rx, self.ry, self.x0, self.y0, self.nx, self.ny = partition(case.nx, case.ny, px, py, rank)
        self.nz = case.nz
        cfg = les.config_from_case(case)
        self._cfg = cfg
        nbytes = C.c_size_t(0)
        les._check(self.lib, None, self.lib.les_dd_workspace_bytes(C.byref(cfg), px, py, C.byref(nbytes)),
                   "les_dd_workspace_bytes")
        self.ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
        base = self.ws.data_ptr()
        base = (base + 255) // 256 * 256
        self.stream = stream or torch.cuda.Stream()
        h = C.c_void_p()
        rc = self.lib.les_dd_create(C.byref(cfg), px, py, self.rx, self.ry, C.c_void_p(base), nbytes.value,
                                    C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != les.LES_OK:
            raise les.LesError(rc, "les_dd_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.les_dd_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def local(self, global_array):
        """This rank's part of a global (nz, ny, nx) array."""
        return global_array[:, self.y0:self.y0 + self.ny, self.x0:self.x0 + self.nx]

    def ops(self, exchange, allreduce):
        """(les_dd_ops, errors): the callbacks around Python callables
        exchange(send, recv, stream) (lists of four byte tensors, None for a
        strip of 0 bytes) and allreduce(values) -> sums; an exception raised
        by either is appended to errors and reported to the library as a
        failure."""
        err = []

        def _ex(ctx, send, recv, nbytes, stream):
            try:
                s = [_view(send[f], nbytes[f]) if nbytes[f] else None for f in range(4)]
                r = [_view(recv[f], nbytes[f]) if nbytes[f] else None for f in range(4)]
                exchange(s, r, self.stream)
                return 0
            except Exception as e:  # reported through the status
                err.append(e)
                return 1

        def _ar(ctx, values, n):
            try:
                v = np.ctypeslib.as_array(values, shape=(n,))
                v[:] = allreduce(v.copy())
                return 0
            except Exception as e:
                err.append(e)
                return 1

        return _Ops(None, _EXCHANGE(_ex), _ALLREDUCE(_ar)), err

    def solve(self, rhs, x, tol: float, maxit: int, exchange, allreduce):
        """les_dd_poisson_solve with Python callables exchange(send, recv,
        stream) (lists of four byte tensors) and allreduce(values) -> sums."""
        from . import les
        ops, err = self.ops(exchange, allreduce)
        it = C.c_int32(0)
        rel = C.c_double(0.0)
        rc = self.lib.les_dd_poisson_solve(self.h, C.cast(C.byref(ops), C.c_void_p), C.c_void_p(rhs.data_ptr()),
                                           C.c_void_p(x.data_ptr()),
                                           float(tol), int(maxit), C.byref(it), C.byref(rel))
        if err:
            raise err[0]
        if rc not in (les.LES_OK, les.LES_ERR_NOT_CONVERGED):
            raise les.LesError(rc, self.lib.les_dd_last_error(self.h).decode())
        return rc, it.value, rel.value


# ---- the decomposed step -----------------------------------------------------

HALO = 2
# fields whose halos each exchange fills (les_dd_halo_exchange)
STEP_FIELDS = ("u", "v", "w", "p", "theta_l", "q_t")   # before the step's thermodynamics
SUB_FIELDS = ("u", "v", "w", "theta_l", "q_t")         # before sub-iterations 1 .. K-1
HAT_FIELDS = ("u_hat", "v_hat")                        # before the right side
PSI_FIELDS = ("psi",)                                  # before the correction


def decomposed_step(sd, K: int, nsteps: int = 1, after=None) -> dict:
    """The order of stages and halo exchanges of one rank's decomposed step
    (Sec. 2.4's stages; Sec. 2.5's exchange before each stencil pass and
    global sums in the solver).  `sd` provides exchange(field names),
    stage(name) and solve() -> stats dict; after(stage, k), if given, is
    called after each stage.  Why these exchanges suffice, with halos two
    nodes deep and every stencil reaching at most two nodes in x and y:

    * BEGIN copies u^n, phi^{n+1/2} and runs the thermodynamics and the
      radiation (pointwise, or along z), so with u v w p theta_l q_t fresh
      everywhere, every field it writes is fresh everywhere;
    * SCALAR and MOMENTUM leave phi^{k+1} and u^ right on the owned nodes;
      the right side's divergence reads u^ one node away along x and v^
      along y (w^ only along z, which is not cut), hence the u^ v^ exchange;
      its App. A term reads psi two nodes away, fresh from the last psi
      exchange;
    * the solve writes psi on the owned nodes; the correction reads psi one
      node away, hence the psi exchange; it leaves u v w fresh but for one
      ring, hence the exchange of u v w and the scalars before the next
      sub-iteration, and p fresh everywhere (p += rho0 psi, pointwise): p is
      exchanged once per step all the same, so that a state set on the owned
      nodes between steps is picked up."""
    tot = {"solves": 0, "iters_total": 0, "iters_max": 0, "not_converged": 0, "res_max": 0.0}

    def done(stage, k):
        if after is not None:
            after(stage, k)

    for _ in range(nsteps):
        sd.exchange(STEP_FIELDS)
        sd.stage("begin")
        done("begin", 0)
        for k in range(K):
            if k:
                sd.exchange(SUB_FIELDS)
            sd.stage("scalar")
            done("scalar", k)
            sd.stage("momentum")
            done("momentum", k)
            sd.exchange(HAT_FIELDS)
            st = sd.solve()
            for key in ("solves", "iters_total", "not_converged"):
                tot[key] += st[key]
            tot["iters_max"] = max(tot["iters_max"], st["iters_max"])
            tot["res_max"] = max(tot["res_max"], st["res_max"])
            done("solve", k)
            sd.exchange(PSI_FIELDS)
            sd.stage("correct")
            done("correct", k)
        sd.stage("end")
        done("end", K - 1)
    return tot


def widened_window(nx: int, ny: int, px: int, py: int, rank: int, halo: int = HALO):
    """(iy, ix): global row and column indices of a rank's widened
    sub-domain (its nodes and `halo` more on each side, wrapped)."""
    rx, ry, x0, y0, nxl, nyl = partition(nx, ny, px, py, rank)
    ix = (x0 - halo + np.arange(nxl + 2 * halo)) % nx
    iy = (y0 - halo + np.arange(nyl + 2 * halo)) % ny
    return iy, ix


class DecomposedSimulation:
    """One rank's sub-domain of the decomposed LES step on the current CUDA
    device: a les handle on the widened sub-domain (les_dd_step_config), the
    sub-domain's decomposed solver (Subdomain), and the halo exchange through
    les_dd_halo_exchange.  exchange(send, recv, stream) and
    allreduce(values) are the same callables as for Subdomain.solve
    (TorchExchange between processes, LocalExchange between threads)."""

    def __init__(self, case, px: int, py: int, rank: int, exchange, allreduce, stream=None):
        from . import les
        if not case.dt > 0:
            raise ValueError("the decomposed step needs a fixed time step (case.dt > 0)")
        self.les = les
        self.sub = Subdomain(case, px, py, rank, stream)
        self.lib = self.sub.lib
        self.case = case
        self.K = case.K
        self.px, self.py, self.rank = px, py, rank
        self.wide = case.replace(nx=self.sub.nx + 2 * HALO, ny=self.sub.ny + 2 * HALO)
        self.sim = les.Simulation(self.wide, stream=self.sub.stream)
        want = les.LesConfig()
        les._check(self.lib, None, self.lib.les_dd_step_config(self.sub.h, C.byref(want)), "les_dd_step_config")
        if (want.nx, want.ny, want.nz) != (self.wide.nx, self.wide.ny, self.wide.nz):
            raise RuntimeError("widened sub-domain differs from the library's")
        self._ops, self._err = self.sub.ops(exchange, allreduce)
        self._opsp = C.cast(C.byref(self._ops), C.c_void_p)
        self.window = widened_window(case.nx, case.ny, px, py, rank)

    def close(self):
        self.sim.close()
        self.sub.close()

    def _raise(self, rc, what, allow=None):
        les = self.les
        if self._err:
            e = self._err[0]
            self._err.clear()
            raise e
        if rc not in (allow or (les.LES_OK,)):
            raise les.LesError(rc, f"{what}: " + self.lib.les_last_error(self.sim.h).decode())

    # -- the steps of decomposed_step ------------------------------------------
    def exchange(self, names) -> None:
        ids = (C.c_int32 * len(names))(*[self.les.FIELDS[n] for n in names])
        rc = self.lib.les_dd_halo_exchange(self.sub.h, self.sim.h, self._opsp, len(names), ids)
        self._raise(rc, "les_dd_halo_exchange")

    def stage(self, name: str) -> None:
        self.sim.stage(name)

    def solve(self) -> dict:
        les = self.les
        st = les.LesStepStats()
        rc = self.lib.les_dd_stage_solve(self.sub.h, self.sim.h, self._opsp, C.byref(st))
        self._raise(rc, "les_dd_stage_solve", (les.LES_OK, les.LES_ERR_NOT_CONVERGED))
        return st.as_dict()

    def step(self, nsteps: int = 1, after=None) -> dict:
        return decomposed_step(self, self.K, nsteps, after)

    # -- fields ------------------------------------------------------------------
    def set_global(self, name: str, value) -> None:
        """Set a field from the global (nz, ny, nx) array (numpy or torch):
        this rank's widened window of it, halos included."""
        iy, ix = self.window
        if isinstance(value, np.ndarray):
            w = value[:, iy][:, :, ix]
        else:
            import torch
            w = value[:, torch.as_tensor(iy, device=value.device)][:, :, torch.as_tensor(ix, device=value.device)]
        self.sim.set(name, w)

    def set_global_state(self, state: dict) -> None:
        for k in ("u", "v", "w", "p", "theta_l", "q_t"):
            if k in state:
                self.set_global(k, state[k])

    def owned(self, name: str) -> np.ndarray:
        """This rank's nodes of a field (nz, ny/py, nx/px), on the host."""
        return self.sim.get(name)[:, HALO:HALO + self.sub.ny, HALO:HALO + self.sub.nx]
