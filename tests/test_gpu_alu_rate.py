"""The measured FMA issue rate behind the FP64 form's ALU roofline
(slh_alu_rate).  Checks what holds on any part: the rates are positive and
finite, FP32 issues at least as fast as FP64, and the FP64 rate is no more
than what the SM count, the maximum SM clock and 128 FMA lanes per SM allow
(a timed kernel that skipped its work would exceed that)."""
import math

import pytest
import torch

import paper_2404_02950_gb300 as slh

pytestmark = pytest.mark.gpu


def test_alu_rate_is_physical():
    fma64 = slh.slh_alu_rate(slh.SLH_F64, 3)
    fma32 = slh.slh_alu_rate(slh.SLH_F32_KAHAN, 3)
    assert math.isfinite(fma64) and fma64 > 0
    assert math.isfinite(fma32) and fma32 > 0
    assert fma32 >= fma64
    props = torch.cuda.get_device_properties(0)
    clock_hz = getattr(props, "clock_rate", 0) * 1e3 or 2.5e9
    # 128 FP32 lanes per SM bound either rate, with 10 % slack for clock reporting
    assert fma32 <= 1.1 * props.multi_processor_count * 128 * clock_hz
    print(f"FP64 {2 * fma64 / 1e12:.4f} TFLOP/s, FP32 {2 * fma32 / 1e12:.2f} TFLOP/s")


def test_alu_rate_rejects_bad_arguments():
    with pytest.raises(slh.SlhError):
        slh.slh_alu_rate(slh.SLH_F32_BF16, 1)
    with pytest.raises(slh.SlhError):
        slh.slh_alu_rate(slh.SLH_F64, 0)
