"""The instruction-rate probes behind the roofline denominators run on the
GPU and return positive rates; the tensor-core probe shows the ceiling the
FP64-accuracy leaf's 128 x 64 x 16 products face: fed from shared memory
alone they issue fewer FLOPs per second than 128 x 128 x 16 products, whose
operand reads per FLOP are a third lower."""
import ctypes

import pytest

from paper_1911_05328_gb300 import mmsr

pytestmark = pytest.mark.gpu


def probe(kind, iters):
    lib = mmsr.load()
    lib.mm_probe_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]
    rate, ms = ctypes.c_double(), ctypes.c_double()
    assert lib.mm_probe_peak(kind, iters, None, ctypes.byref(rate), ctypes.byref(ms)) == mmsr.MM_OK
    return rate.value, ms.value


@pytest.mark.parametrize("kind,iters", [(0, 2000), (1, 2000), (2, 200), (3, 2000), (4, 500), (5, 500)])
def test_probe_runs(kind, iters):
    rate, ms = probe(kind, iters)
    assert rate > 0 and ms > 0


def test_wider_products_issue_faster():
    probe(4, 200)
    probe(5, 200)
    n64 = probe(4, 2000)[0]
    n128 = probe(5, 2000)[0]
    assert n128 > 1.2 * n64, (n64, n128)
