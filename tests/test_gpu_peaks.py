"""Measured pipe peaks (gb_measure_peak): the denominators of the roofline
fractions.  Each loop must report a rate within the range the unit counts
and clocks of a GB300 allow (152 SMs, at most 2.07 GHz): FP64 FMA 4 flop
per clock per SM (1.26 TFLOP/s), FP32 FMA 256 (80.5 TFLOP/s), dense 16-bit
tensor MMA about 2.25 PFLOP/s nominal, TF32 half of that.  The lower ends
allow for the clock under load."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RANGES_TFLOPS = {"dfma": (0.6, 1.4), "ffma": (40.0, 90.0), "dmma": (0.05, 1.4),
                 "tc_bf16": (900.0, 2600.0), "tc_f16": (900.0, 2600.0),
                 "tc_tf32": (400.0, 1300.0), "dfma_dmma": (0.5, 2.8)}


@pytest.fixture(scope="module")
def h():
    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    hd = binding.Handle(0)
    yield hd
    hd.close()


@pytest.mark.parametrize("kind", sorted(RANGES_TFLOPS))
def test_peak_in_range(h, kind):
    lo, hi = RANGES_TFLOPS[kind]
    v = h.measure_peak(kind) / 1e12
    assert lo <= v <= hi, f"{kind}: {v:.2f} TFLOP/s"


def test_bad_kind_rejected(h):
    import ctypes
    v = ctypes.c_double()
    assert h.lib.gb_measure_peak(h.h, 7, ctypes.byref(v)) == -2
