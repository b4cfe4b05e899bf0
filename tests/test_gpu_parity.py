"""GPU parity: the CUDA path through the C ABI against the CPU oracle, bit for
bit (all results are integers).  Inputs come from the seeded generator."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_18974_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def ctx(ms):
    c = ms.MaxSquare(0)
    yield c
    c.close()


DEV = "cuda:0"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def bits_dev(a, n, pad=0, ldw=None):
    w = gen.pack_bits(a, n, ldw=ldw, pad_value=pad)
    return torch.from_numpy(w.view(np.int32)).to(DEV)


def run_all_paths(ctx, a, check_map=True, pads=(0, 1)):
    """Every entry point on matrix a (uint8, m x n) against the oracle."""
    m, n = a.shape
    (K, r, c), dref = oracle.dp(a)
    exp = [K, r, c, 0]
    x = to_dev(a)
    assert ctx.max_square(x).cpu().tolist() == exp, ("u8", m, n)
    if check_map:
        dp, res = ctx.dp_map(x)
        assert res.cpu().tolist() == exp, ("u8 map", m, n)
        assert np.array_equal(dp.cpu().numpy(), dref), ("u8 map values", m, n)
    for pad in pads:
        w = bits_dev(a, n, pad=pad)
        assert ctx.max_square(w, n=n).cpu().tolist() == exp, ("bits", m, n, pad)
        if check_map:
            dp, res = ctx.dp_map(w, n=n)
            assert res.cpu().tolist() == exp, ("bits map", m, n, pad)
            assert np.array_equal(dp.cpu().numpy(), dref), ("bits map values", m, n, pad)
    return K, r, c


SHAPES = [(1, 1), (1, 7), (7, 1), (2, 2), (31, 33), (32, 32), (33, 31), (64, 65), (100, 127),
          (129, 128), (255, 257), (300, 512), (257, 513), (70, 992), (40, 993), (33, 1505),
          (520, 700), (1000, 1100)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("p", [0.3, 0.8, 0.95])
def test_random_shapes(ctx, shape, p):
    m, n = shape
    a = gen.bernoulli_u8(m, n, p, seed=m * 1000 + n + int(p * 100))
    run_all_paths(ctx, a)


@pytest.mark.parametrize("band_rows", [32, 64, 96])
def test_many_bands_and_planted_squares_cross_tiles(ctx, band_rows):
    """Small bands force many tiles; planted squares larger than the 32-cell
    halo straddle tile rows and strips, so the exact fix-up runs."""
    ctx.set_tuning(band_rows=band_rows)
    try:
        rng = np.random.default_rng(band_rows)
        for t in range(6):
            m, n = int(rng.integers(200, 700)), int(rng.integers(400, 2200))
            a = gen.bernoulli_u8(m, n, 0.9, seed=100 + t)
            for s in [40, 75, int(rng.integers(33, min(m, n)))]:
                r0, c0 = int(rng.integers(0, m - s + 1)), int(rng.integers(0, n - s + 1))
                a[r0:r0 + s, c0:c0 + s] = 1
            run_all_paths(ctx, a, pads=(1,))
    finally:
        ctx.set_tuning(band_rows=0)


@pytest.mark.parametrize("lane_cols", [1, 2, 4, 8, 16, 32])
def test_every_lane_width(ctx, lane_cols):
    """Each tile width forced on ragged shapes (edge chunks, several strips,
    several bands), with planted squares above the halo crossing strip and
    band edges: every entry point and both formats against the oracle."""
    ctx.set_tuning(band_rows=64, lane_cols=lane_cols)
    try:
        rng = np.random.default_rng(500 + lane_cols)
        W = 32 * lane_cols
        for t, (m, n) in enumerate([(150, 3 * W - 40 + 7), (97, W + 1), (300, 2 * W + 33),
                                    (70, max(W - 5, 1))]):
            a = gen.bernoulli_u8(m, n, 0.85, seed=7000 + 10 * lane_cols + t)
            s = min(m, n, 70)
            if s > 33:
                r0 = int(rng.integers(0, m - s + 1))
                c0 = min(max(W - s // 2, 0), n - s)
                a[r0:r0 + s, c0:c0 + s] = 1
            run_all_paths(ctx, a, check_map=(m * n <= 400_000), pads=(1,))
    finally:
        ctx.set_tuning()


def test_wide_matrix_automatic_lane_width(ctx):
    """Wide size-only inputs take 32 columns per lane by default; the dp map
    keeps 16.  Both must agree with the oracle across many strips."""
    m, n = 400, 6000
    a = gen.bernoulli_u8(m, n, 0.9, seed=8123)
    a[100:190, 2000:2090] = 1
    a[300:340, 5950:5990] = 1
    run_all_paths(ctx, a, check_map=True, pads=(0, 1))


def test_large_boxes_shared_by_block_teams(ctx):
    """Large flagged boxes are shared by teams of blocks (one matrix alone,
    and several in a batch): side and witness against the oracle."""
    mats, exps = [], []
    for t, (m, n, s) in enumerate([(6000, 6000, 1500), (2048, 2048, 1400), (1800, 2000, 900)]):
        a = gen.bernoulli_u8(m, n, 0.9, seed=9100 + t)
        r0, c0 = (m - s) // 3, (n - s) // 2
        a[r0:r0 + s, c0:c0 + s] = 1
        exp = list(oracle.dp(a, want_map=False)[0]) + [0]
        assert exp[0] >= s
        x = to_dev(a)
        assert ctx.max_square(x).cpu().tolist() == exp, (m, n, "u8")
        w = bits_dev(a, n, pad=1)
        assert ctx.max_square(w, n=n).cpu().tolist() == exp, (m, n, "bits")
        mats += [x, (w, n)]
        exps += [exp, exp]
    assert ctx.batch(mats).cpu().tolist() == exps


def test_dp_map_levels_by_cluster(ctx):
    """A large matrix's dp-map levels are built by a cluster of blocks: the
    whole map against the oracle, with the flagged box spanning most rows."""
    m, n, s = 6000, 6000, 2100
    a = gen.bernoulli_u8(m, n, 0.92, seed=9200)
    a[300:300 + s, 3000:3000 + s] = 1
    a[3500:3500 + 900, 100:100 + 900] = 1
    want, ref = oracle.dp(a, want_map=True)
    assert want[0] == s
    dp, res = ctx.dp_map(to_dev(a))
    assert res.cpu().tolist() == list(want) + [0]
    assert np.array_equal(dp.cpu().numpy(), ref)
    dpb, resb = ctx.dp_map(bits_dev(a, n, pad=3), n=n)
    assert resb.cpu().tolist() == list(want) + [0]
    assert np.array_equal(dpb.cpu().numpy(), ref)


def test_squares_on_tile_edges(ctx):
    ctx.set_tuning(band_rows=64)
    try:
        n = 2000
        for (r0, c0, s) in [(0, 0, 64), (63, 511, 33), (64, 512, 40), (31, 480, 100),
                            (100, 991, 34), (127, 1471, 65), (190, 960, 200)]:
            a = gen.bernoulli_u8(400, n, 0.6, seed=r0 + c0 + s)
            a[r0:r0 + s, c0:c0 + s] = 1
            run_all_paths(ctx, a, pads=(0,))
    finally:
        ctx.set_tuning(band_rows=0)


def test_narrow_matrices_with_large_squares(ctx):
    """Narrow matrices use short lane chunks; squares above the halo at odd
    columns make the fix-up start at unaligned columns (both formats, alone
    and batched)."""
    mats, exps = [], []
    for i, (m, n) in enumerate([(633, 94), (400, 37), (300, 61), (500, 128), (700, 200),
                                (260, 33), (900, 255)]):
        a = gen.bernoulli_u8(m, n, 0.3, seed=900 + i)
        s = min(m, n) - 3
        c0 = 1 + (i % 3)
        a[m - s - 2:m - 2, c0:c0 + s] = 1
        exp = list(oracle.dp(a, want_map=False)[0]) + [0]
        assert exp[0] == s
        run_all_paths(ctx, a, pads=(1,))
        mats += [to_dev(a), (bits_dev(a, n, pad=1), n)]
        exps += [exp, exp]
    assert ctx.batch(mats).cpu().tolist() == exps


@pytest.mark.parametrize("shape", [(1, 1), (1, 600), (600, 1), (5, 9), (512, 512), (700, 1500),
                                   (2000, 1300)])
def test_closed_forms(ctx, shape):
    m, n = shape
    s = min(m, n)
    ones = np.ones((m, n), dtype=np.uint8)
    K = run_all_paths(ctx, ones, check_map=(m * n <= 1_000_000))
    assert K == (s, s - 1, s - 1)
    zeros = np.zeros((m, n), dtype=np.uint8)
    assert run_all_paths(ctx, zeros, check_map=False) == (0, -1, -1)
    one = zeros.copy()
    one[m // 2, n // 3] = 1
    assert run_all_paths(ctx, one, check_map=False) == (1, m // 2, n // 3)
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    chk = ((ii + jj) % 2 == 1).astype(np.uint8)
    if m * n > 1:
        exp = (1, 0, 1) if n > 1 else (1, 1, 0)
        assert run_all_paths(ctx, chk, check_map=False) == exp


def test_all_ones_large_uses_fixup_everywhere(ctx):
    m, n = 4096, 3000
    x = torch.ones((m, n), dtype=torch.uint8, device=DEV)
    assert ctx.max_square(x).cpu().tolist() == [3000, 2999, 2999, 0]
    dp, res = ctx.dp_map(x)
    assert res.cpu().tolist() == [3000, 2999, 2999, 0]
    ii = torch.arange(m, device=DEV).view(-1, 1)
    jj = torch.arange(n, device=DEV).view(1, -1)
    assert torch.equal(dp, torch.minimum(ii, jj).to(torch.int32) + 1)


def test_empty_matrices(ctx):
    for shp in [(0, 5), (5, 0), (0, 0)]:
        x = torch.zeros(shp, dtype=torch.uint8, device=DEV)
        assert ctx.max_square(x).cpu().tolist() == [0, -1, -1, 0]
        dp, res = ctx.dp_map(x)
        assert res.cpu().tolist() == [0, -1, -1, 0]


def test_nonzero_bytes_and_strides(ctx):
    rng = np.random.default_rng(3)
    a = (rng.random((300, 900)) < 0.9).astype(np.uint8)
    a[50:120, 200:270] = 1
    vals = a * rng.integers(1, 256, size=a.shape).astype(np.uint8)
    (K, r, c), dref = oracle.dp(a)
    # ld not a multiple of 16, and a column-offset view (unaligned base)
    big = torch.zeros((300, 1003), dtype=torch.uint8, device=DEV)
    big[:, 3:903] = to_dev(vals)
    view = big[:, 3:903]
    assert ctx.max_square(view).cpu().tolist() == [K, r, c, 0]
    dp, res = ctx.dp_map(view)
    assert np.array_equal(dp.cpu().numpy(), dref)
    # dp map written with a padded row stride
    dpbig = torch.full((300, 907), -7, dtype=torch.int32, device=DEV)
    ctx.dp_map(view, dp=dpbig[:, :900])
    assert np.array_equal(dpbig[:, :900].cpu().numpy(), dref)
    assert (dpbig[:, 900:] == -7).all()
    # packed rows with extra words per row (ldw > ceil(n/32)) and pad bits set
    w = bits_dev(a, 900, pad=1, ldw=40)
    assert ctx.max_square(w, n=900).cpu().tolist() == [K, r, c, 0]


@pytest.mark.parametrize("tile_kind,lane_cols", [(1, 4), (1, 8), (1, 16), (1, 32), (2, 0)])
def test_aligned_rows_with_ragged_last_chunk(ctx, tile_kind, lane_cols):
    """16-byte-aligned rows (a padded row stride) whose width is not a multiple
    of 16: the last chunk of each row is copied with a partial source size.
    The padding bytes are ones, and against the right edge sits a block of
    ones s rows high and s - 3 columns wide: a copy that read past column n
    would see an s-square there."""
    ctx.set_tuning(band_rows=64, lane_cols=lane_cols, tile_kind=tile_kind)
    try:
        views, exps = [], []
        for t, n in enumerate([17, 100, 527, 1031, 2047, 3003]):
            m = 230
            a = gen.bernoulli_u8(m, n, 0.8, seed=9100 + t)
            s = min(60, n)
            a[40:40 + s, n - max(s - 3, 1):n] = 1
            ld = (n + 15) // 16 * 16 + 16
            big = torch.ones((m, ld), dtype=torch.uint8, device=DEV)
            big[:, :n] = to_dev(a)
            x = big[:, :n]
            (K, r, c), dref = oracle.dp(a)
            exp = [K, r, c, 0]
            assert ctx.max_square(x).cpu().tolist() == exp, (n, tile_kind, lane_cols)
            dp, res = ctx.dp_map(x)
            assert res.cpu().tolist() == exp, (n, "map")
            assert np.array_equal(dp.cpu().numpy(), dref), (n, "map values")
            views.append(x)
            exps.append(exp)
        for kind in (0, 1, 2):
            ctx.set_tuning(band_rows=64, tile_kind=kind)
            assert ctx.batch(views).cpu().tolist() == exps, ("batch", kind)
    finally:
        ctx.set_tuning()


def test_dp_map_store_alignments(ctx):
    """The dp map through each store path: 32-byte rows (256-bit stores),
    16-byte rows (128-bit stores) and unaligned rows (scalar stores), with
    cells outside the map left untouched."""
    a = gen.bernoulli_u8(200, 1500, 0.9, seed=77)
    a[20:110, 600:690] = 1
    (K, r, c), dref = oracle.dp(a)
    x = to_dev(a)
    for off, ld in [(0, 1504), (4, 1504), (1, 1503), (8, 1512)]:
        buf = torch.full((200 * ld + 64,), -3, dtype=torch.int32, device=DEV)
        view = buf[off:off + 200 * ld].view(200, ld)[:, :1500]
        dp, res = ctx.dp_map(x, dp=view)
        assert res.cpu().tolist() == [K, r, c, 0], (off, ld)
        assert np.array_equal(view.cpu().numpy(), dref), (off, ld)
        rest = buf.cpu().numpy().copy()
        idx = off + np.arange(200)[:, None] * ld + np.arange(1500)[None, :]
        rest[idx.ravel()] = -3
        assert (rest == -3).all(), (off, ld)


def test_generated_c1_with_dp_map(ctx):
    """256 x 256, Bernoulli(0.5), seed 0: side, witness and the full dp map."""
    a = gen.bernoulli_u8(256, 256, 0.5, seed=0)
    K = run_all_paths(ctx, a)
    assert oracle.freq(a) == K


def test_batch_mixed_shapes_and_formats(ctx):
    rng = np.random.default_rng(11)
    mats, exps, singles = [], [], []
    for i in range(60):
        m = int(np.exp(rng.uniform(np.log(1), np.log(900))))
        n = int(np.exp(rng.uniform(np.log(1), np.log(1500))))
        p = float(rng.choice(np.arange(1, 10) / 10))
        a = gen.bernoulli_u8(m, n, p, seed=500 + i)
        if i % 2 and min(m, n) > 1:
            s = int(rng.integers(1, min(m, n) + 1))
            r0, c0 = gen.plant_pos(500 + i, m, n, s)
            a[r0:r0 + s, c0:c0 + s] = 1
        (K, r, c), _ = oracle.dp(a, want_map=False)
        exps.append([K, r, c, 0])
        if i % 3 == 0:
            mats.append((bits_dev(a, n, pad=i % 2), n))
        else:
            mats.append(to_dev(a))
    out = ctx.batch(mats).cpu().tolist()
    assert out == exps
    # each result alone equals its result in the mix
    for i, item in enumerate(mats[:20]):
        res = ctx.max_square(*item) if isinstance(item, tuple) else ctx.max_square(item)
        assert res.cpu().tolist() == out[i]
    # repeated call (job table reused) and CUDA-graph capture of the same call
    assert ctx.batch(mats).cpu().tolist() == exps
    outbuf = torch.empty((len(mats), 4), dtype=torch.int32, device=DEV)
    ctx.batch(mats, out=outbuf)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ctx.batch(mats, out=outbuf)
    outbuf.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert outbuf.cpu().tolist() == exps


def plane_words(m, n):
    """Words of one small-matrix plane: rows at an odd pitch, rounded to 4."""
    w = (n + 31) // 32
    return (m * (w | 1) + 3) // 4 * 4


@pytest.mark.parametrize("limit,w", [(512, 1), (2048, 1), (6144, 3), (14320, 5), (28672, 7)])
def test_batch_small_class_boundaries(ctx, limit, w):
    """Matrices whose plane is exactly a size class's limit and one row more
    (the next class, or bitplane tiles past the largest), 32w columns and
    32w - 5 (a ragged last chunk), uint8 in aligned rows and packed; random
    cells with a planted square against the right edge.  Every result equals
    the oracle's, in one batch and in a batch of one."""
    m_at = limit // w
    assert plane_words(m_at, 32 * w) == limit and plane_words(m_at + 1, 32 * w) > limit
    mats, exps = [], []
    for k, (m, n) in enumerate([(m_at, 32 * w), (m_at + 1, 32 * w), (m_at, 32 * w - 5),
                                (m_at + 1, 32 * w - 5)]):
        a = gen.bernoulli_u8(m, n, 0.8, seed=9300 + 10 * w + k)
        s = min(m, n, 20 + 3 * k)
        a[m // 3:m // 3 + s, n - s:n] = 1
        (K, r, c), _ = oracle.dp(a, want_map=False)
        ld = (n + 15) // 16 * 16
        big = torch.zeros((m, ld), dtype=torch.uint8, device=DEV)
        big[:, :n] = to_dev(a)
        mats.append(big[:, :n])
        exps.append([K, r, c, 0])
        mats.append((bits_dev(a, n, pad=1), n))
        exps.append([K, r, c, 0])
    assert ctx.batch(mats).cpu().tolist() == exps
    for item, exp in zip(mats, exps):
        one = ctx.batch([item, item]).cpu().tolist()
        assert one == [exp, exp]


def test_invalid_arguments(ctx, ms):
    x = torch.zeros((10, 10), dtype=torch.uint8, device=DEV)
    desc = ms.describe(x)
    desc.ld = 5
    assert ms.lib().ms_max_square(ctx._h, ms.ctypes.byref(desc), x.data_ptr(), None) == 1
    desc = ms.describe(x)
    desc.fmt = 7
    assert ms.lib().ms_max_square(ctx._h, ms.ctypes.byref(desc), x.data_ptr(), None) == 1
    desc = ms.describe(x)
    desc.m = 70000
    assert ms.lib().ms_max_square(ctx._h, ms.ctypes.byref(desc), x.data_ptr(), None) == 6
    desc = ms.describe(x)  # (refused before any access: the buffer is never read)
    desc.m, desc.n, desc.ld = 1, 1 << 31, 1 << 31
    assert ms.lib().ms_max_square(ctx._h, ms.ctypes.byref(desc), x.data_ptr(), None) == 6
    desc = ms.describe(x)
    assert ms.lib().ms_max_square(ctx._h, ms.ctypes.byref(desc), None, None) == 1
    # tunings out of range are refused and leave the context's tuning as it was
    before = ctx.get_tuning()
    for bad in (dict(tile_kind=3), dict(tile_kind=-1), dict(lane_cols=3), dict(band_rows=-1),
                dict(band_rows=16385), dict(packed_path=2)):
        with pytest.raises(ms.MSError):
            ctx.set_tuning(**bad)
    assert ctx.get_tuning() == before


@pytest.fixture
def packed_ctx(ctx):
    ctx.set_tuning(packed_path=1)
    yield ctx
    ctx.set_tuning(packed_path=0)


@pytest.mark.parametrize("shape", [(1, 1), (1, 40), (40, 1), (31, 33), (64, 1024), (100, 1025),
                                   (257, 3000), (1000, 700), (33, 2050)])
@pytest.mark.parametrize("p", [0.2, 0.7, 0.95])
def test_packed_search_random(packed_ctx, shape, p):
    """The bitplane doubling / binary search (packed size-only path)."""
    m, n = shape
    a = gen.bernoulli_u8(m, n, p, seed=7 * m + n + int(100 * p))
    (K, r, c), _ = oracle.dp(a, want_map=False)
    for pad in (0, 1):
        w = gen.pack_bits(a, n, ldw=((n + 31) // 32 + 3) // 4 * 4, pad_value=pad)
        x = torch.from_numpy(w.view(np.int32)).to(DEV)
        assert packed_ctx.max_square(x, n=n).cpu().tolist() == [K, r, c, 0], (shape, p, pad)


def test_packed_search_planted_and_closed_forms(packed_ctx):
    rng = np.random.default_rng(21)
    cases = []
    for t in range(8):
        m, n = int(rng.integers(50, 1500)), int(rng.integers(50, 2500))
        a = gen.bernoulli_u8(m, n, 0.8, seed=300 + t)
        s = int(rng.integers(20, min(m, n) + 1))
        r0, c0 = int(rng.integers(0, m - s + 1)), int(rng.integers(0, n - s + 1))
        a[r0:r0 + s, c0:c0 + s] = 1
        cases.append(a)
    cases += [np.ones((300, 500), np.uint8), np.ones((777, 64), np.uint8),
              np.zeros((200, 300), np.uint8)]
    one = np.zeros((90, 3000), np.uint8)
    one[55, 2047] = 1
    cases.append(one)
    for a in cases:
        m, n = a.shape
        (K, r, c), _ = oracle.dp(a, want_map=False)
        w = gen.pack_bits(a, n, ldw=((n + 31) // 32 + 3) // 4 * 4, pad_value=1)
        x = torch.from_numpy(w.view(np.int32)).to(DEV)
        assert packed_ctx.max_square(x, n=n).cpu().tolist() == [K, r, c, 0], (m, n)
        # the same matrix through the tile path
        packed_ctx.set_tuning(packed_path=0)
        assert packed_ctx.max_square(x, n=n).cpu().tolist() == [K, r, c, 0], (m, n)
        packed_ctx.set_tuning(packed_path=1)


def test_autotune_then_results_unchanged(ctx):
    """The autotuner only changes launch parameters: results stay exact."""
    rng = np.random.default_rng(31)
    mats, exps = [], []
    for i in range(40):
        m, n = int(rng.integers(16, 700)), int(rng.integers(16, 900))
        a = gen.bernoulli_u8(m, n, 0.85, seed=700 + i)
        if i % 4 == 0:
            s = int(rng.integers(1, min(m, n) + 1))
            a[:s, n - s:] = 1
        exps.append(list(oracle.dp(a, want_map=False)[0]) + [0])
        mats.append(to_dev(a) if i % 2 else (bits_dev(a, n), n))
    chosen = ctx.autotune(mats)
    assert chosen["band_rows"] in (0, 32, 64, 128, 256, 512, 1024)
    assert ctx.batch(mats).cpu().tolist() == exps
    one = gen.bernoulli_u8(600, 3000, 0.9, seed=77)
    one[100:400, 1000:1300] = 1
    exp1 = list(oracle.dp(one, want_map=False)[0]) + [0]
    w = bits_dev(one, 3000, ldw=96)
    chosen1 = ctx.autotune([(w, 3000)])
    assert chosen1["packed_path"] in (0, 1)
    assert ctx.max_square(w, n=3000).cpu().tolist() == exp1
    assert ctx.get_tuning()["band_rows"] == 0  # explicit tuning untouched


def test_bounded_wait_times_out_and_context_recovers(ctx):
    """Failure detection without a fault: the first fix-up strip withholds its
    carries (a test hook), the next strip's wait gives up after about a second,
    the matrix reports MS_ERR_TIMEOUT and the next call is exact again."""
    a = gen.bernoulli_u8(700, 2000, 0.6, seed=91)
    a[100:600, 300:1200] = 1  # a 500-square: the fix-up box spans several strips
    (K, r, c), _ = oracle.dp(a, want_map=False)
    x = to_dev(a)
    ctx.set_tuning(test_hold_carries=1)
    try:
        # the dp-map fix-up walks the box in strips that pass carries
        _, res = ctx.dp_map(x)
        res = res.cpu().tolist()
    finally:
        ctx.set_tuning()
    assert res[3] == 4  # MS_ERR_TIMEOUT
    dp, res2 = ctx.dp_map(x)
    assert res2.cpu().tolist() == [K, r, c, 0]
    assert ctx.max_square(x).cpu().tolist() == [K, r, c, 0]
