"""Ensembles of independent members stepped together (les_ensemble_step) and
the autotuner: every member reaches exactly the state of the same member run
alone, and the autotuner leaves the state it tunes on unchanged."""
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


def _members():
    return inputs.ensemble(4, seed=3, xy=(32, 48, 64), zs=(16, 24))


def test_ensemble_matches_solo_runs(les_mod):
    cases = _members()
    assert len({(c.nx, c.nz) for c in cases}) > 1          # uneven grids
    ens = les_mod.Ensemble(cases)
    ens.set_states([inputs.initial_state(c) for c in cases])
    stats = ens.step(2)
    assert all(s["not_converged"] == 0 and s["solves"] == 2 * c.K for s, c in zip(stats, cases))
    torch.cuda.synchronize()
    for c, m in zip(cases, ens.members):
        solo = les_mod.Simulation(c)
        solo.set_state(inputs.initial_state(c))
        solo.step(2)
        for f in ("u", "v", "w", "p", "theta_l", "q_t"):
            assert np.array_equal(m.get(f), solo.get(f)), (c.name, f)
        solo.close()
    ens.close()


def test_ensemble_tune_restores_states(les_mod):
    """tune() times the members stepped together and one after another from
    the same states and puts the states back: stepping in the mode it chose,
    and in the other mode from a fresh ensemble, ends bit-identical to each
    member run alone."""
    cases = _members()
    ens = les_mod.Ensemble(cases)
    ens.set_states([inputs.initial_state(c) for c in cases])
    res = ens.tune(steps=1)
    assert set(res["ms_per_step"]) == {"together", "one_after_another"}
    assert res["together"] == ens.together
    chosen = ens.together
    other = les_mod.Ensemble(cases, together=not chosen)
    other.set_states([inputs.initial_state(c) for c in cases])
    for e in (ens, other):
        stats = e.step(2)
        assert all(st["not_converged"] == 0 for st in stats)
    torch.cuda.synchronize()
    for i, c in enumerate(cases):
        solo = les_mod.Simulation(c)
        solo.set_state(inputs.initial_state(c))
        solo.step(2)
        for f in ("u", "v", "w", "p", "theta_l", "q_t"):
            ref = solo.get(f)
            assert np.array_equal(ens.members[i].get(f), ref), (c.name, f, chosen)
            assert np.array_equal(other.members[i].get(f), ref), (c.name, f, not chosen)
        solo.close()
    ens.close()
    other.close()


@pytest.mark.parametrize("share", [2, 4])
def test_ensemble_shared_sms_matches_solo_runs(les_mod, share):
    """Members capped at 1/share of the SMs solve concurrently; each member
    still ends bit-identical to the same member run alone with the same
    tuning (its grid, hence its order of sums, is the same)."""
    cases = _members()
    ens = les_mod.Ensemble(cases, share=share)
    ens.set_states([inputs.initial_state(c) for c in cases])
    stats = ens.step(2)
    assert all(s["not_converged"] == 0 for s in stats)
    torch.cuda.synchronize()
    for c, m in zip(cases, ens.members):
        solo = les_mod.Simulation(c)
        solo.set_state(inputs.initial_state(c))
        solo.set_tuning(cg_max_blocks=m.tuning()["cg_max_blocks"])
        solo.step(2)
        for f in ("u", "v", "w", "p", "theta_l", "q_t"):
            assert np.array_equal(m.get(f), solo.get(f)), (c.name, f)
        solo.close()
    ens.close()


def test_ensemble_member_against_oracle(les_mod):
    from oracle import Oracle
    c = _members()[1]
    ens = les_mod.Ensemble([c, _members()[0]])
    st = inputs.initial_state(c)
    ens.set_states([st, inputs.initial_state(_members()[0])])
    ens.step(1)
    ref = Oracle(c.replace(precision=64), st)
    ref.step(1)
    sim = ens.members[0]
    for f in ("u", "v", "theta_l", "q_t"):
        a, b = sim.get(f), ref.get(f)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5, f
    ens.close()


def test_ensemble_rejects_repeated_handles(les_mod):
    c = _members()[0]
    sim = les_mod.Simulation(c)
    hs = (C.c_void_p * 2)(sim.h.value, sim.h.value)
    failed = C.c_int32(0)
    rc = sim.lib.les_ensemble_step(hs, 2, 1, None, C.byref(failed))
    assert rc == les_mod.LES_ERR_INVALID_ARG
    sim.close()


def test_autotune_keeps_the_state(les_mod):
    c = _members()[2]
    sim = les_mod.Simulation(c)
    sim.set_state(inputs.initial_state(c))
    sim.step(1)
    before = {f: sim.get(f) for f in ("u", "v", "w", "p", "theta_l", "q_t")}
    res = les_mod.autotune(sim)
    assert res["tuning"] in [dict(x) for x in les_mod.AUTOTUNE_CANDIDATES]
    assert len(res["ms_per_step"]) == len(les_mod.AUTOTUNE_CANDIDATES)
    for f, v in before.items():
        assert np.array_equal(sim.get(f), v), f
    # and it keeps stepping with the chosen tuning
    st = sim.step(1)
    assert st["not_converged"] == 0
    sim.close()
