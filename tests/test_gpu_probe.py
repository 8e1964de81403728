"""Throughput probes of the units that bound the kernel product (MUFU exp2, FFMA, and
tcgen05.mma in the product's shapes): each returns a rate within physical limits and
leaves no error behind."""
import pytest

pytestmark = pytest.mark.gpu

# nominal dense BF16 tensor peak of the part (2.25 PFLOP/s); a probe cannot exceed it by
# more than clock and rounding slack
BF16_NOMINAL = 2.25e15


@pytest.mark.parametrize("what", ["mma_ss_n128", "mma_ss_n256", "mma_ss_n128_tmem_ld", "mma_ts_n80"])
def test_mma_probes_are_within_the_tensor_peak(native, what):
    rate = native.probe_throughput(what)
    assert 0.05 * BF16_NOMINAL < rate < 1.15 * BF16_NOMINAL, (what, rate)
    assert native.sync_status() == native.OK


def test_tf32_mma_probe_is_within_the_tf32_peak(native):
    """TF32 tensor flops: half the BF16 rate per instruction shape (1.1 PFLOP/s nominal)."""
    rate = native.probe_throughput("mma_ss_n128_tf32")
    assert 0.05 * BF16_NOMINAL / 2 < rate < 1.15 * BF16_NOMINAL / 2, rate
    assert native.sync_status() == native.OK


def test_unit_probes_are_positive(native):
    assert native.probe_throughput("ex2") > 1e11
    assert native.probe_throughput("ffma") > 1e12
    assert native.probe_throughput("rsqrt") > 1e11
    # FP64 runs far below FP32 on this part (about 1.25 TFLOP/s nominal)
    assert 1e10 < native.probe_throughput("dfma") < 1e14
    assert native.sync_status() == native.OK
