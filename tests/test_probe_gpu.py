"""The FP32 FMA throughput probe (the measured roofline denominator of the FP32
kernels) returns a throughput consistent with the device's FP32 lanes and clock."""
import pytest
import torch


@pytest.mark.gpu
def test_fp32_fma_probe_is_within_the_lane_bound():
    from paper_1803_01215_gb300 import binding
    props = torch.cuda.get_device_properties(0)
    # 128 FP32 lanes per SM, 2 flops per FMA, at most 2.2 GHz
    bound = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    scalar = binding.probe_fp32_fma(4000, packed=False)
    packed = binding.probe_fp32_fma(4000, packed=True)
    assert 0.3 * bound < scalar <= 1.05 * bound
    assert 0.3 * bound < packed <= 2.1 * bound


@pytest.mark.gpu
def test_fp32_fma_probe_rejects_bad_arguments():
    from paper_1803_01215_gb300 import binding
    with pytest.raises(binding.HJError):
        binding.probe_fp32_fma(0)
