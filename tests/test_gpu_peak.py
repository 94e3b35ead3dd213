"""The arithmetic peaks the ALU roofline is taken against, measured on the
device (tbr_measure_peak): each rate lies between 0.5x and 1.05x of the rate
the SM count, the per-SM unit counts and the current SM clock imply, so that
a fraction of a measured peak cannot hide a wrong denominator."""
import pytest
import torch

from paper_2609_08722_b300 import tbr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,per_sm_clock", [("ffma2", 128 * 2), ("ffma", 128 * 2), ("ex2", 32), ("rcp", 16)])
def test_measured_peak_is_plausible(kind, per_sm_clock):
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    rate, ms = tbr.measure_peak(kind, iters=100000)
    # FP32: 128 lanes x 2 FLOPs per SM per clock; MUFU: 16 results per SM per clock,
    # 32 for ex2 (measured: B300 runs ex2.approx at twice the other MUFU ops' rate);
    # a clock between 1.0 and 2.1 GHz
    lo, hi = sms * per_sm_clock * 1.0e9 * 0.5, sms * per_sm_clock * 2.1e9 * 1.05
    print(f"{kind}: {rate / 1e12:.2f} T/s in {ms:.1f} ms")
    assert ms > 1.0
    assert lo <= rate <= hi
