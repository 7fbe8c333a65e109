"""les_measure_fma: the FP32 and FP64 FMA rates of the device (the ALU bounds
of the issue-bound kernels), and its argument checks."""
import ctypes as C

import pytest

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


def test_fma_rates_are_positive_and_fp64_is_slower(les_mod):
    r32 = les_mod.measure_fma(32, 200)
    r64 = les_mod.measure_fma(64, 10)
    assert r32["tflops"] > 0 and r32["ms"] > 0
    assert r64["tflops"] > 0 and r64["ms"] > 0
    # the work is the same FMAs per launch trip in both precisions; FP32 has
    # the wider pipes on every GPU this library targets
    assert r32["tflops"] > r64["tflops"]


def test_fma_rate_refuses_bad_arguments(les_mod):
    lib = les_mod.load_library()
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    assert lib.les_measure_fma(None, 16, 10, C.byref(tf), C.byref(ms)) == les_mod.LES_ERR_INVALID_ARG
    assert lib.les_measure_fma(None, 32, 0, C.byref(tf), C.byref(ms)) == les_mod.LES_ERR_INVALID_ARG
    assert lib.les_measure_fma(None, 64, 10, None, C.byref(ms)) == les_mod.LES_ERR_INVALID_ARG
