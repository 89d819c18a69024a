"""Pins of the oracle's FP8 E4M3 rounding (the FP8 depth plane of the atlas,
the reduced-precision form of the probe maps): codes derived by hand from
the format, ties to even, saturation, and agreement with PyTorch's own
float8_e4m3fn cast over every in-range float32 sampled densely."""
import numpy as np
import pytest


def test_hand_codes(orc):
    cases = {0.0: 0x00, 1.0: 0x38, 0.5: 0x30, 2.0: 0x40, 448.0: 0x7E, 2.0 ** -6: 0x08, 2.0 ** -9: 0x01,
             7 * 2.0 ** -9: 0x07, 1.125: 0x39, 1.875: 0x3F, 240.0: 0x77, -1.0: 0xB8, -448.0: 0xFE}
    for x, c in cases.items():
        assert int(orc.fp8_e4m3_bits(np.float32(x))) == c, (x, hex(c))


def test_ties_to_even_and_saturation(orc):
    # 1.0625 lies halfway between 1.0 (mantissa 0) and 1.125 (mantissa 1)
    assert int(orc.fp8_e4m3_bits(np.float32(1.0625))) == 0x38
    # 1.1875 lies halfway between 1.125 (1) and 1.25 (2): to the even one
    assert int(orc.fp8_e4m3_bits(np.float32(1.1875))) == 0x3A
    # halfway between the subnormals 2^-9 and 2^-8 (1.5 * 2^-9): to 2^-8
    assert int(orc.fp8_e4m3_bits(np.float32(1.5 * 2.0 ** -9))) == 0x02
    # half of the smallest subnormal rounds to zero (even)
    assert int(orc.fp8_e4m3_bits(np.float32(2.0 ** -10))) == 0x00
    for big in (449.0, 464.0, 1e6, np.inf):
        assert int(orc.fp8_e4m3_bits(np.float32(big))) == 0x7E
    assert int(orc.fp8_e4m3_bits(np.float32(np.nan))) == 0x7F


def test_matches_torch_float8_cast(orc):
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(0, 448, 200000), np.exp(rng.uniform(np.log(2.0 ** -12), np.log(448), 200000)),
                        np.arange(0, 448, 1 / 64.0)]).astype(np.float32)
    x = np.concatenate([x, -x])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(orc.fp8_e4m3_bits(x), ref)
