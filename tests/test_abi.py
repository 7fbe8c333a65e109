"""The C ABI library loads and exports every symbol declared in include/les.h
(no compute call: these run without a GPU)."""
import ctypes as C
import os
import re

import pytest

from paper_2301_04698_gb300 import build as B
from paper_2301_04698_gb300 import inputs, les

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return les.load_library()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "les.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(les_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in les.h but not exported"
    assert set(declared) == set(les.EXPORTED)


def test_config_struct_matches_abi(lib):
    cfg = les.LesConfig()
    lib.les_config_default(C.byref(cfg), 8, 9, 10)
    assert cfg.struct_size == C.sizeof(les.LesConfig)
    assert (cfg.nx, cfg.ny, cfg.nz) == (8, 9, 10)
    # Table 1 defaults
    assert cfg.cs == 0.18 and cfg.pr == 0.4 and cfg.sc == 0.4
    assert cfg.theta0 == 290.0 and cfg.p00 == 1e5 and cfg.f_cor == 7.62e-5


def test_workspace_bytes_and_validation(lib):
    for case in (inputs.tgv(32), inputs.cbl(24, 20, 16, precision=64), inputs.cbl()):
        cfg = les.config_from_case(case)
        n = C.c_size_t(0)
        assert lib.les_workspace_bytes(C.byref(cfg), C.byref(n)) == les.LES_OK
        es = 8 if case.precision == 64 else 4
        assert n.value >= 28 * case.n * es
        assert n.value % 256 == 0
    bad = les.config_from_case(inputs.tgv(8))
    bad.nx = 2
    n = C.c_size_t(0)
    assert lib.les_workspace_bytes(C.byref(bad), C.byref(n)) == les.LES_ERR_INVALID_ARG
    bad = les.config_from_case(inputs.tgv(8))
    bad.struct_size = 4
    assert lib.les_workspace_bytes(C.byref(bad), C.byref(n)) == les.LES_ERR_INVALID_ARG
    bad = les.config_from_case(inputs.tgv(8, solver="jacobi", op="wide"))
    assert lib.les_workspace_bytes(C.byref(bad), C.byref(n)) == les.LES_ERR_INVALID_ARG
    h = C.c_void_p()
    good = les.config_from_case(inputs.tgv(8))
    # a NULL workspace is rejected before any device call
    assert lib.les_init(C.byref(good), None, None, 0, None, C.byref(h)) == les.LES_ERR_INVALID_ARG
    assert lib.les_status_string(3) == b"Poisson solve did not converge"
    assert lib.les_last_error(None) == b"no handle"


def test_ensemble_members_are_seeded_and_uneven():
    from paper_2301_04698_gb300 import inputs
    a = inputs.ensemble(16, seed=1)
    b = inputs.ensemble(16, seed=1)
    c = inputs.ensemble(16, seed=2)
    assert [(x.nx, x.ny, x.nz, x.shf, x.seed) for x in a] == [(x.nx, x.ny, x.nz, x.shf, x.seed) for x in b]
    assert [(x.nx, x.nz) for x in a] != [(x.nx, x.nz) for x in c]
    assert len({(x.nx, x.nz) for x in a}) > 4
    for x in a:
        assert x.nx in (64, 96, 128, 160, 192) and x.nz in (64, 96, 128) and x.nx == x.ny
        assert 0.5 * 15.0 <= x.shf < 1.5 * 15.0 and 0.5 * 3.75e-6 <= x.subs_div < 1.5 * 3.75e-6
    assert len({inputs.cbl_draws(x)["zi"] for x in a}) == 16   # every member its own inversion
