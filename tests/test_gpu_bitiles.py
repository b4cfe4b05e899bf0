"""GPU parity of the bitplane tile pass (size-only single calls, tile_kind 2)
against the CPU oracle, bit for bit: ragged shapes, every largest side up to
past the 33-cell exact limit, ties, squares on band and strip edges, bytes
other than 0/1, strided and unaligned inputs, padded packed rows."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
STRIP = 992  # counted columns of a 1024-column tile after the first strip


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_18974_gb300 as m
    m.build()
    c = m.MaxSquare(0)
    c.set_tuning(tile_kind=2)
    yield c
    c.close()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def bits_dev(a, n, pad=0, ldw=None):
    w = gen.pack_bits(a, n, ldw=ldw, pad_value=pad)
    return torch.from_numpy(w.view(np.int32)).to(DEV)


def check(ctx, a, pads=(0, 1), what=""):
    m, n = a.shape
    (K, r, c), _ = oracle.dp(a, want_map=False)
    exp = [K, r, c, 0]
    assert ctx.max_square(to_dev(a)).cpu().tolist() == exp, ("u8", m, n, what)
    for pad in pads:
        got = ctx.max_square(bits_dev(a, n, pad=pad), n=n).cpu().tolist()
        assert got == exp, ("bits", m, n, pad, what)
    return K, r, c


SHAPES = [(1, 1), (1, 7), (7, 1), (2, 2), (31, 33), (32, 32), (33, 31), (64, 65), (100, 127),
          (129, 128), (255, 257), (300, 512), (257, 513), (70, 992), (40, 993), (33, 1505),
          (520, 700), (1000, 1100), (97, 2017), (2100, 90),
          # rows of 16-byte multiples: whole 1024-column tile rows arrive by bulk copies
          (300, 1024), (97, 2048), (520, 2976), (45, 3008)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("p", [0.3, 0.8, 0.95])
def test_random_shapes(ctx, shape, p):
    m, n = shape
    check(ctx, gen.bernoulli_u8(m, n, p, seed=31 * m + n + int(p * 100)))


@pytest.mark.parametrize("band_rows", [0, 32, 64, 160])
def test_every_side_up_to_past_the_exact_limit(ctx, band_rows):
    """A sparse background with one planted s-square: K = s for every s from
    1 to 40, so the threshold test climbs through every level, and from 33 on
    the exact fix-up takes over."""
    ctx.set_tuning(tile_kind=2, band_rows=band_rows)
    try:
        rng = np.random.default_rng(40 + band_rows)
        for s in range(1, 41):
            m, n = int(rng.integers(s, 400)), int(rng.integers(s, 2500))
            if s % 2:
                n = max(16 * ((n + 15) // 16), 1024)  # bulk-copied rows
            a = gen.bernoulli_u8(m, n, 0.15, seed=1000 * s + band_rows)
            r0, c0 = int(rng.integers(0, m - s + 1)), int(rng.integers(0, n - s + 1))
            a[r0:r0 + s, c0:c0 + s] = 1
            K, _, _ = check(ctx, a, pads=(1,), what=s)
            assert K >= s
    finally:
        ctx.set_tuning(tile_kind=2)


def test_ties_first_corner_in_row_major_order(ctx):
    """Equal largest squares in different tiles and on the same row: the
    witness is the first bottom-right corner in row-major order."""
    ctx.set_tuning(tile_kind=2, band_rows=64)
    try:
        for s in (5, 17, 32, 33, 48):
            a = gen.bernoulli_u8(700, 3000, 0.1, seed=s)
            for (r1, c1) in [(400, 2900), (400, 1500), (650, 100), (130, 2500)]:
                a[r1 - s + 1:r1 + 1, c1 - s + 1:c1 + 1] = 1
            K, r, c = check(ctx, a, what=s)
            assert (K, r, c) == (s, 130, 2500)
    finally:
        ctx.set_tuning(tile_kind=2)


def test_squares_on_band_and_strip_edges(ctx):
    ctx.set_tuning(tile_kind=2, band_rows=64)
    try:
        n = 4 * STRIP + 100
        for (r0, c0, s) in [(0, 0, 33), (63, 1023, 33), (64, 1024, 32), (31, STRIP + 31, 34),
                            (100, 2 * STRIP + 32 - 17, 40), (127, 3 * STRIP, 31),
                            (190, n - 64, 64), (0, n - 33, 33)]:
            a = gen.bernoulli_u8(400, n, 0.7, seed=r0 + c0 + s)
            a[r0:r0 + s, c0:c0 + s] = 1
            check(ctx, a, pads=(0,), what=(r0, c0, s))
    finally:
        ctx.set_tuning(tile_kind=2)


def test_closed_forms(ctx):
    for (m, n) in [(1, 1), (33, 33), (40, 2000), (1500, 70), (700, 1100)]:
        s = min(m, n)
        assert check(ctx, np.ones((m, n), dtype=np.uint8), pads=(0,)) == (s, s - 1, s - 1)
        zeros = np.zeros((m, n), dtype=np.uint8)
        assert check(ctx, zeros, pads=(1,)) == (0, -1, -1)
        one = zeros.copy()
        one[m // 2, n // 3] = 1
        assert check(ctx, one, pads=(1,)) == (1, m // 2, n // 3)
        ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
        if m * n > 1:
            chk = ((ii + jj) % 2 == 1).astype(np.uint8)
            exp = (1, 0, 1) if n > 1 else (1, 1, 0)
            assert check(ctx, chk, pads=(0,)) == exp


def test_bytes_above_one_strides_and_unaligned_bases(ctx):
    """Nonzero bytes other than 1 (the 0/1 shortcut must notice and redo the
    tile), a row stride that is not a multiple of 16 and a column-offset view
    (byte loads), and packed rows with spare words and pad bits set."""
    rng = np.random.default_rng(5)
    a = (rng.random((500, 2100)) < 0.9).astype(np.uint8)
    a[50:120, 1000:1070] = 1
    a[300:330, 10:40] = 1
    (K, r, c), _ = oracle.dp(a, want_map=False)
    vals = a * rng.integers(1, 256, size=a.shape).astype(np.uint8)
    assert ctx.max_square(to_dev(vals)).cpu().tolist() == [K, r, c, 0]
    big = torch.zeros((500, 2111), dtype=torch.uint8, device=DEV)
    big[:, 5:2105] = to_dev(vals)
    assert ctx.max_square(big[:, 5:2105]).cpu().tolist() == [K, r, c, 0]
    big[:, 5:2105] = to_dev(a)
    assert ctx.max_square(big[:, 5:2105]).cpu().tolist() == [K, r, c, 0]
    w = bits_dev(a, 2100, pad=1, ldw=70)
    assert ctx.max_square(w, n=2100).cpu().tolist() == [K, r, c, 0]
    # 16-byte rows (bulk copies) with bytes above one, and a 16-byte-aligned
    # view whose last tile reaches past the matrix (lane copies there)
    b = (rng.random((400, 3072)) < 0.9).astype(np.uint8)
    b[10:90, 2000:2080] = 1
    (K, r, c), _ = oracle.dp(b, want_map=False)
    vb = b * rng.integers(1, 256, size=b.shape).astype(np.uint8)
    assert ctx.max_square(to_dev(vb)).cpu().tolist() == [K, r, c, 0]
    assert ctx.max_square(to_dev(b)).cpu().tolist() == [K, r, c, 0]
    big = torch.zeros((400, 3104), dtype=torch.uint8, device=DEV)
    big[:, 16:3040] = to_dev(b[:, :3024])
    (K, r, c), _ = oracle.dp(b[:, :3024], want_map=False)
    assert ctx.max_square(big[:, 16:3040]).cpu().tolist() == [K, r, c, 0]


def test_large_matrix_automatic_choice(ctx):
    """The automatic choice: bitplane tiles once the matrix fills the GPU's
    tile warps with bands of 64 rows or more (checked on a 26000 x 8192 matrix
    with a planted square on zeros, whose answer is known), the dp
    recurrence below that; both, and the forced kinds, match the oracle."""
    import paper_2503_18974_gb300 as m
    c = m.MaxSquare(0)
    try:
        big = torch.zeros((26000, 8192), dtype=torch.uint8, device=DEV)
        big[20000:20150, 5000:5150] = 1
        big[20100:20200, 7000:7099] = 1
        c.profile_start()
        assert c.max_square(big).cpu().tolist() == [150, 20149, 5149, 0]
        p = c.profile_stop()
        assert p.tile_launches == 1 and p.bit_tile_launches == 1
        del big
        a = gen.bernoulli_u8(3000, 5000, 0.9, seed=99)
        a[2000:2100, 100:200] = 1
        (K, r, cc), _ = oracle.dp(a, want_map=False)
        x = to_dev(a)
        c.profile_start()
        assert c.max_square(x).cpu().tolist() == [K, r, cc, 0]
        assert c.profile_stop().bit_tile_launches == 0
        c.set_tuning(tile_kind=2)
        assert c.max_square(x).cpu().tolist() == [K, r, cc, 0]
        c.set_tuning(tile_kind=1)
        assert c.max_square(x).cpu().tolist() == [K, r, cc, 0]
        b = gen.bernoulli_u8(2500, 4000, 0.9, seed=98)
        (K, r, cc), _ = oracle.dp(b, want_map=False)
        c.set_tuning(tile_kind=0)
        assert c.max_square(to_dev(b)).cpu().tolist() == [K, r, cc, 0]
        assert c.max_square(bits_dev(b, 4000, pad=1), n=4000).cpu().tolist() == [K, r, cc, 0]
    finally:
        c.close()


@pytest.mark.parametrize("kind,band_rows", [(0, 0), (2, 64), (2, 0)])
def test_batch_with_bitplane_tiles(ctx, kind, band_rows):
    """Batches with tile kind 2 run every matrix as bitplane tiles in the
    persistent launch (kind 0: the dp recurrence's pairs); planted squares
    below, at and above the exact limit hand their S_33 rows to the batched
    fix-up.  Every result against the oracle, and alone vs in the mix."""
    import paper_2503_18974_gb300 as m
    c = m.MaxSquare(0)
    try:
        c.set_tuning(tile_kind=kind, band_rows=band_rows)
        rng = np.random.default_rng(77 + kind + band_rows)
        mats, exps = [], []
        for i in range(24):
            mm = int(rng.integers(40, 900))
            nn = int(rng.choice([int(rng.integers(20, 700)), int(rng.integers(768, 3100))]))
            a = gen.bernoulli_u8(mm, nn, float(rng.choice([0.3, 0.8, 0.93])), seed=900 + i)
            s = min(mm, nn, int(rng.choice([20, 33, 34, 70, 300])))
            r0, c0 = int(rng.integers(0, mm - s + 1)), int(rng.integers(0, nn - s + 1))
            a[r0:r0 + s, c0:c0 + s] = 1
            (K, r, cc), _ = oracle.dp(a, want_map=False)
            exps.append([K, r, cc, 0])
            mats.append((bits_dev(a, nn, pad=1), nn) if i % 3 == 0 else to_dev(a))
        out = c.batch(mats).cpu().tolist()
        assert out == exps
        assert c.batch(mats).cpu().tolist() == exps  # the table reused
        for i, item in enumerate(mats[:6]):
            res = c.max_square(*item) if isinstance(item, tuple) else c.max_square(item)
            assert res.cpu().tolist() == exps[i]
    finally:
        c.close()
