"""Host-side packing of the BF16 tensor storage (the binding's marshalling
of SLH_F32_BF16 states): round to nearest even, pairs in (low, high)
order, exact widening back."""
import numpy as np

import paper_2404_02950_gb300 as slh


def test_pack_roundtrip_and_rounding():
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0], dtype=np.float32)
    b = np.array([3.0, 1.0 + 2 ** -9, 1.0 - 2 ** -10, 1e-3, -0.0], dtype=np.float32)
    z = np.zeros(5, np.float32)
    slots = slh.pack_bf16_fields([z] * 4 + [a, b] + [z] * 10)
    assert len(slots) == slh.SLH_SLOTS_BF16
    back = slh.unpack_bf16_fields(slots)
    # ties go to the even mantissa: 1 + 2^-8 -> 1, 1 + 3 2^-8 -> 1 + 2^-6
    assert np.array_equal(back[4], np.array([1.0, 1.0, 1.0 + 4 * 2 ** -8, -2.5, 0.0], np.float32))
    assert back[5][0] == 3.0 and back[5][1] == 1.0 and back[5][2] == 1.0
    assert abs(back[5][3] - 1e-3) <= 2 ** -9 * 1e-3 and np.signbit(back[5][4])
    # the first field of a pair sits in the low half of its slot
    w = slots[4].view(np.uint32)
    assert w[0] == (0x3F80 | (0x4040 << 16))
    # the scalar slots pass through unchanged, widening is exact
    r = np.random.default_rng(0).standard_normal(5).astype(np.float32)
    again = slh.unpack_bf16_fields(slh.pack_bf16_fields([r] * 16))
    assert np.array_equal(again[0], r)
    assert np.array_equal(slh.unpack_bf16_fields(slh.pack_bf16_fields(again))[7], again[7])
