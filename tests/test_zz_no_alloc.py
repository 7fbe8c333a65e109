"""The allocation-free Poisson solve (les_poisson_solve_static), called through
the C ABI, against the handle-based les_poisson_solve on the same inputs.

It exists for callers that cannot allocate device memory (a plug-in whose
host application owns all device memory through its own pool allocator, or a
latency-bound loop that must not call cudaMalloc / cudaFree).  Its scratch is
one static device array shared by every call, so two calls in a row are
checked: the second must not see leftovers of the first.  This file is
collected last on purpose.
"""
import ctypes as C

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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _static_solve(les_mod, lib, case, b, tol, maxit, rho0=None, x=None):
    cfg = les_mod.config_from_case(case)
    err = C.create_string_buffer(256)
    if x is None:
        x = torch.zeros_like(b)
    it = C.c_int32(0)
    rel = C.c_double(0.0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.les_poisson_solve_static(C.byref(cfg), C.c_void_p(rho0.data_ptr()) if rho0 is not None else None,
                                      C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), tol, maxit,
                                      C.c_void_p(stream), C.byref(it), C.byref(rel), err, len(err))
    torch.cuda.synchronize()
    return rc, x, it.value, rel.value, err.value


def _case(nx, ny, nz, precision, walls, op="compact", solver="cg"):
    return inputs.Case(name="static", nx=nx, ny=ny, nz=nz, dx=35.0, dy=35.0, dz=10.0, walls=walls,
                       precision=precision, init="zero", physics=(), op=op, solver=solver,
                       rho0_const=None if walls else 1.0)


@pytest.mark.parametrize("precision,walls,op", [(64, True, "compact"), (32, True, "compact"),
                                                (64, False, "wide")])
def test_static_solve_matches_handle_solve(les_mod, precision, walls, op):
    case = _case(40, 36, 20, precision, walls, op)
    tol = 1e-10 if precision == 64 else 1e-6
    dt = torch.float64 if precision == 64 else torch.float32
    sim = les_mod.Simulation(case)
    rho0 = torch.ones(case.nz, dtype=dt, device="cuda")
    lib = sim.lib
    for call, seed in enumerate((11, 12)):
        # a right side in the operator's range (D(rho0 G) has more than the
        # constant in its null space on an even periodic grid)
        xt = torch.from_numpy(inputs.uniform(seed, 0, case.n, -1, 1).reshape(case.shape)).to("cuda", dt)
        b = sim.apply_poisson(xt, op)
        x_ref = torch.zeros_like(b)
        rc_ref, it_ref, res_ref = sim.poisson_solve(b, x_ref, tol, 5000)
        rc, x, it, rel, msg = _static_solve(les_mod, lib, case, b, tol, 5000, rho0)
        assert rc == les_mod.LES_OK, msg
        # the handle's solver may be a different (persistent) CG kernel whose
        # sums round in another order: the same iterates to within rounding
        assert rel <= tol and abs(it - it_ref) <= (1 if precision == 64 else 3)
        assert _rel(x.cpu().double().numpy(), x_ref.cpu().double().numpy()) < (1e-9 if precision == 64 else 1e-5), call
    sim.close()


def test_static_weighted_jacobi_matches_handle_solve(les_mod):
    """The Jacobi branch keeps its second iterate in the array and reports the
    buffer holding the answer through the control block: the same answer
    and iteration count as the handle's weighted Jacobi, twice in a row."""
    case = _case(16, 12, 8, 64, True, solver="jacobi")
    sim = les_mod.Simulation(case)
    for seed in (21, 22):
        xt = torch.from_numpy(inputs.uniform(seed, 0, case.n, -1, 1).reshape(case.shape)).to("cuda", torch.float64)
        b = sim.apply_poisson(xt, "compact")
        x_ref = torch.zeros_like(b)
        rc_ref, it_ref, res_ref = sim.poisson_solve(b, x_ref, 1e-4, 20000)
        rc, x, it, rel, msg = _static_solve(les_mod, sim.lib, case, b, 1e-4, 20000)
        assert rc == les_mod.LES_OK, msg
        assert it == it_ref and rel <= 1e-4
        assert _rel(x.cpu().numpy(), x_ref.cpu().numpy()) < 1e-12
    sim.close()


def test_static_solve_allocates_nothing_and_keeps_no_state(les_mod):
    """A call leaves the device's free memory unchanged once the library's
    module is loaded on the device (the first call of a process may load it,
    so each grid gets one call first); and a solve on a large grid followed by
    one on a smaller grid (whose vectors then start inside the large grid's
    leftovers) still matches the handle's solve."""
    lib = les_mod.load_library()
    results = []
    for dims in ((96, 80, 32), (40, 36, 20)):
        case = _case(*dims, 32, True)
        sim = les_mod.Simulation(case)
        xt = torch.from_numpy(inputs.uniform(31, 0, case.n, -1, 1).reshape(case.shape)).to("cuda", torch.float32)
        b = sim.apply_poisson(xt, "compact")
        x_ref = torch.zeros_like(b)
        sim.poisson_solve(b, x_ref, 1e-6, 5000)
        rc, _, _, _, msg = _static_solve(les_mod, lib, case, b, 1e-6, 5000)
        assert rc == les_mod.LES_OK, msg
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc, x, it, rel, msg = _static_solve(les_mod, lib, case, b, 1e-6, 5000, x=x)
        free1 = torch.cuda.mem_get_info()[0]
        assert rc == les_mod.LES_OK, msg
        assert free1 == free0
        results.append(_rel(x.cpu().double().numpy(), x_ref.cpu().double().numpy()))
        sim.close()
    assert max(results) < 1e-5


def test_static_solve_rejects_oversized_grids(les_mod):
    case = inputs.Case(name="big", nx=128, ny=128, nz=64, dx=1.0, dy=1.0, dz=1.0, precision=64, init="zero",
                       physics=())
    cfg = les_mod.config_from_case(case)
    lib = les_mod.load_library()
    err = C.create_string_buffer(256)
    it = C.c_int32(0)
    rel = C.c_double(0.0)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.les_poisson_solve_static(C.byref(cfg), None, C.c_void_p(dummy.data_ptr()),
                                      C.c_void_p(dummy.data_ptr()), 1e-8, 10, None, C.byref(it),
                                      C.byref(rel), err, len(err))
    assert rc == les_mod.LES_ERR_INVALID_ARG
    assert b"exceeds the static scratch limit" in err.value
