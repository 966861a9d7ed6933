"""GPU tests of the measurement probes: the tcgen05 rate of each operand kind the sweep
kernels use and the per-SM bulk-copy ingest from L2 are measured and plausible."""
import pytest

from gpu_helpers import pim

pytestmark = pytest.mark.gpu


def test_tensor_probe_rates_are_ordered():
    P = pim()
    bf16 = P.pim_probe_tensor("bf16", 4000)
    fp8 = P.pim_probe_tensor("fp8", 4000)
    e2m1 = P.pim_probe_tensor("e2m1", 4000)
    assert 100.0 < bf16 < 10000.0
    assert fp8 > bf16 and e2m1 > bf16


def test_ingest_probe_and_argument_checks():
    P = pim()
    own = P.pim_probe_ingest(32768, 400, shared=False)
    shared = P.pim_probe_ingest(16384, 400, shared=True)
    assert 1.0 < own < 1000.0 and 1.0 < shared < 1000.0
    with pytest.raises(P.PimError):
        P.pim_probe_ingest(100, 10)
    with pytest.raises(P.PimError):
        P.pim_probe_tensor("int8", 10)
