"""rbm_fp32_fma_peak: the measured FP32 FMA throughput that bounds the
direct O(N^2) sum.  Eight independent chains per thread on every SM must
come within a plausible range of the nominal rate (152 SMs x 128 FP32 lanes
x 2 flop x the SM clock): well above half of it (the loop is not starved)
and not above it by more than clock variation allows, for scalar FMA; the
packed two-lane form is reported beside it."""
import pytest

import paper_1812_10575_gb300 as rbm
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def test_fma_peak_scalar_and_packed_plausible():
    torch = torch_cuda()
    props = torch.cuda.get_device_properties(0)
    # nominal at the GB300's 2070 MHz maximum SM clock, per SM 128 FP32 lanes
    nominal = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    scalar = rbm.rbm_fp32_fma_peak(False)
    packed = rbm.rbm_fp32_fma_peak(True)
    assert 0.5 * nominal < scalar < 1.1 * nominal, (scalar, nominal)
    assert 0.5 * nominal < packed < 2.2 * nominal, (packed, nominal)
