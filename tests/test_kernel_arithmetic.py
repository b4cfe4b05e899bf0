"""CPU pins of the arithmetic facts the kernels rely on, checked exhaustively
in numpy (no GPU, no oracle): the multiply that packs eight 0/1 bytes into
eight bits, the exactness and ordering of small integers in fp16 (the
size-only dp-recurrence tiles keep dp in fp16 halves), and the decode of an
fp16 integer's bits."""
import numpy as np


def test_eight_bytes_to_eight_bits_by_one_multiply():
    # q = r0 + 16 r1 holds column i in bit 8i and column 4+i in bit 8i+4
    # (r0, r1 = four 0/1 bytes each); times 0x00204081 the product's bits
    # 21..28 are the eight columns in order, with no carry
    for pattern in range(256):
        cells = [(pattern >> b) & 1 for b in range(8)]
        r0 = sum(cells[i] << (8 * i) for i in range(4))
        r1 = sum(cells[4 + i] << (8 * i) for i in range(4))
        q = (r0 + 16 * r1) & 0xFFFFFFFF
        y = (q * 0x00204081) & 0xFFFFFFFF
        assert (y >> 21) & 0xFF == pattern, pattern


def test_small_integers_in_fp16():
    v = np.arange(0, 2049, dtype=np.int64)
    h = v.astype(np.float16)
    assert np.array_equal(h.astype(np.int64), v)  # every integer up to 2048 is exact
    bits = h.view(np.uint16).astype(np.int64)
    assert np.all(np.diff(bits) > 0)  # non-negative values order like their bit patterns
    # one + min(up, left, diag): the window's dp never exceeds 1024 (a tile is at
    # most 1024 columns wide), and v*m + v with v in {0, 1} is exact there
    one = np.float16(1.0)
    for m in range(0, 1024):
        mm = np.float16(m)
        got = np.float16(np.float32(one) * np.float32(mm) + np.float32(one))
        assert int(got) == m + 1
        assert np.float16(np.float32(0.0) * np.float32(mm) + np.float32(0.0)) == 0


def test_fp16_integer_decode():
    # value of the fp16 bits h of a whole number: (1024 + mantissa) >> (25 - exponent)
    for v in range(0, 2048):
        h = int(np.float16(v).view(np.uint16))
        dec = 0 if h == 0 else (1024 | (h & 1023)) >> (25 - (h >> 10))
        assert dec == v, v
    # the halo constant: 32.0 is 0x5000, 1.0 is 0x3C00
    assert int(np.float16(32.0).view(np.uint16)) == 0x5000
    assert int(np.float16(1.0).view(np.uint16)) == 0x3C00
