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
    fills the four halo strips (torch tensors on the group's device)."""

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
        ops = []
        local = []
        for face, side, halo in TRAVEL:
            dst = self.nb[side]                 # where this rank's strip goes
            src = self.nb[OPPOSITE[side]]       # whose strip fills the halo
            if dst == self.rank and src == self.rank:
                local.append((halo, face))
                continue
            ops.append(dist.P2POp(dist.isend, send[face], dst, self.group))
            ops.append(dist.P2POp(dist.irecv, recv[halo], src, self.group))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
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

    def solve(self, rhs, x, tol: float, maxit: int, exchange, allreduce):
        """les_dd_poisson_solve with Python callables exchange(send, recv,
        stream) (lists of four byte tensors) and allreduce(values) -> sums."""
        from . import les
        err = []

        def _ex(ctx, send, recv, nbytes, stream):
            try:
                s = [_view(send[f], nbytes[f]) for f in range(4)]
                r = [_view(recv[f], nbytes[f]) for f in range(4)]
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

        ops = _Ops(None, _EXCHANGE(_ex), _ALLREDUCE(_ar))
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
