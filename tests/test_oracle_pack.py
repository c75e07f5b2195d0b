"""Pins the oracle's little-endian bit-stream encodings and object sizes."""
import numpy as np
import pytest


def py_pack(vals, bits):
    acc = 0
    for i, v in enumerate(vals):
        acc |= int(v) << (bits * i)
    return acc.to_bytes((len(vals) * bits + 7) // 8, "little")


@pytest.mark.parametrize("bits", [3, 4, 6, 10, 13, 18, 20])
def test_pack_matches_integer_bitstream(orc, bits):
    rng = np.random.default_rng(bits)
    vals = rng.integers(0, 1 << bits, 256).astype(np.uint32)
    packed = orc.pack_bits(vals, bits)
    assert packed == py_pack(vals, bits)
    assert len(packed) == 256 * bits // 8
    assert np.array_equal(orc.unpack_bits(packed, 256, bits), vals)


def test_sizes_follow_table1_widths(orc):
    # pk = rho + k*320; sk = 3*32 + (l+k)*eta_bytes + k*416; sig = 32 + l*z_bytes + omega + k
    assert orc.sizes(2) == (32 + 4 * 320, 96 + 8 * 96 + 4 * 416, 32 + 4 * 576 + 80 + 4)
    assert orc.sizes(3) == (32 + 6 * 320, 96 + 11 * 128 + 6 * 416, 32 + 5 * 640 + 55 + 6)
    assert orc.sizes(5) == (32 + 8 * 320, 96 + 15 * 96 + 8 * 416, 32 + 7 * 640 + 75 + 8)
    assert orc.sizes(2) == (1312, 2528, 2420)
    assert orc.sizes(3) == (1952, 4000, 3293)
    assert orc.sizes(5) == (2592, 4864, 4595)


def test_bad_level_rejected(orc):
    with pytest.raises(ValueError):
        orc.sizes(4)
