"""les_prefetch_states: states uploaded ahead on a copy stream are the ones
the following steps start from, bit for bit as if uploaded with
les_set_states just before each step; at most two may be pending."""
import numpy as np
import pytest

from paper_2301_04698_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAMES = ("u", "v", "w", "p", "theta_l", "q_t")


@pytest.fixture(scope="module")
def les_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_04698_gb300 import build, les
    build.build()
    les.load_library()
    return les


def _host_state(case, seed):
    st = inputs.initial_state(case)
    for i, k in enumerate(("u", "v", "w")):
        st[k] = st[k] + 0.1 * inputs.uniform(seed, 50 + i, case.n, -1, 1).reshape(case.shape)
    return {k: torch.from_numpy(np.ascontiguousarray(st[k], dtype=np.float32)).pin_memory() for k in NAMES}


@pytest.mark.parametrize("shape", [(64, 16, 12), (40, 12, 9)])
def test_prefetched_states_step_like_uploaded_ones(les_mod, shape):
    case = inputs.tgv(32, nxyz=shape, precision=32, steps_tol=1e-6)
    states = [_host_state(case, s) for s in (1, 2, 3)]
    # reference: each state uploaded (synchronously) right before its step
    ref = les_mod.Simulation(case)
    want = []
    for st in states:
        ref.set_many_from_host(st)
        ref.step(1)
        want.append({k: ref.get(k) for k in NAMES})
    sim = les_mod.Simulation(case)
    copy = torch.cuda.Stream()
    staging = [torch.empty(len(NAMES) * case.n, dtype=torch.float32, device="cuda") for _ in range(2)]
    sim.prefetch_from_host(states[0], staging[0], copy)
    sim.prefetch_from_host(states[1], staging[1], copy)
    with pytest.raises(les_mod.LesError) as e:          # a third one while two are pending
        sim.prefetch_from_host(states[2], staging[0], copy)
    assert e.value.status == les_mod.LES_ERR_STATE
    for q in range(3):
        if q == 1:   # staging[0] again, after the step that consumed it was enqueued
            sim.prefetch_from_host(states[2], staging[0], copy)
        sim.step(1)
        for k in NAMES:
            assert np.array_equal(sim.get(k), want[q][k]), (q, k)
    ref.close()
    sim.close()


def test_prefetch_refuses_bad_arguments(les_mod):
    """A misaligned staging buffer, a repeated field, a bad field id and no
    fields are refused before anything is copied."""
    import ctypes as C
    case = inputs.tgv(32, nxyz=(64, 16, 12), precision=32, steps_tol=1e-6)
    sim = les_mod.Simulation(case)
    host = _host_state(case, 1)
    copy = torch.cuda.Stream()
    staging = torch.empty(len(NAMES) * case.n + 4, dtype=torch.float32, device="cuda")
    ids = (C.c_int32 * 2)(les_mod.FIELDS["u"], les_mod.FIELDS["u"])
    ptrs = (C.c_void_p * 2)(host["u"].data_ptr(), host["v"].data_ptr())
    stream = C.c_void_p(copy.cuda_stream)
    lib = sim.lib
    misaligned = C.c_void_p(staging.data_ptr() + 4)
    good = C.c_void_p(staging.data_ptr())
    one = (C.c_int32 * 1)(les_mod.FIELDS["u"])
    assert lib.les_prefetch_states(sim.h, 1, one, ptrs, misaligned, stream) == les_mod.LES_ERR_INVALID_ARG
    assert lib.les_prefetch_states(sim.h, 2, ids, ptrs, good, stream) == les_mod.LES_ERR_INVALID_ARG
    bad = (C.c_int32 * 1)(999)
    assert lib.les_prefetch_states(sim.h, 1, bad, ptrs, good, stream) == les_mod.LES_ERR_INVALID_ARG
    assert lib.les_prefetch_states(sim.h, 0, one, ptrs, good, stream) == les_mod.LES_ERR_INVALID_ARG
    # nothing is pending: a step runs from the state set before
    sim.set_state({k: v.numpy() for k, v in host.items()})
    sim.step(1)
    sim.close()
