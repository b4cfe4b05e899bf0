"""All largest squares (every corner with dp == K) through the C ABI against
the oracle's list: the set must be equal (the device lists in unspecified
order, so both sides are sorted), the count exact even when the capacity is
smaller, and the side and witness equal to ms_max_square's."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_18974_gb300 as m
    m.build()
    c = m.MaxSquare(0)
    yield c
    c.close()


def check(ctx, a, fmt_bits=False):
    m, n = a.shape
    (K, r, c), want = oracle.all_max(a)
    if fmt_bits:
        x = torch.from_numpy(gen.pack_bits(a, n, pad_value=1).view(np.int32)).to(DEV)
        res, got = ctx.all_max_squares(x, n=n, capacity=8)
    else:
        x = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
        res, got = ctx.all_max_squares(x, capacity=8)
    assert res.cpu().tolist() == [K, r, c, 0], (m, n)
    got = sorted(tuple(p) for p in got.cpu().tolist())
    assert got == [tuple(p) for p in want.tolist()], (m, n, K, len(got), len(want))
    return K, len(want)


@pytest.mark.parametrize("shape", [(1, 1), (31, 33), (100, 127), (300, 512), (257, 1100),
                                   (700, 2500)])
@pytest.mark.parametrize("p", [0.5, 0.9])
def test_random_small_side(ctx, shape, p):
    """K at most the halo: the corners come from the second tile pass."""
    a = gen.bernoulli_u8(shape[0], shape[1], p, seed=shape[0] * 7 + shape[1] + int(p * 10))
    for bits in (False, True):
        check(ctx, a, bits)


def test_planted_equal_squares_large_side(ctx):
    """K above the halo: several planted squares of the same side (one
    touching the matrix edge) are listed by the bitplane fix-up."""
    for t, (m, n, s) in enumerate([(400, 900, 50), (1200, 1500, 130), (3000, 2600, 301)]):
        a = gen.bernoulli_u8(m, n, 0.6, seed=5000 + t)
        a[10:10 + s, 20:20 + s] = 1
        a[m - s:, n - s:] = 1
        a[m // 2:m // 2 + s, n // 3:n // 3 + s] = 1
        K, cnt = check(ctx, a)
        assert K == s and cnt >= 3
        check(ctx, a, True)


def test_all_ones_many_corners(ctx):
    for m, n in [(64, 64), (300, 200), (40, 1000), (1500, 1400)]:
        K, cnt = check(ctx, np.ones((m, n), dtype=np.uint8))
        s = min(m, n)
        assert K == s and cnt == (m - s + 1) * (n - s + 1)


def test_empty_and_zero(ctx):
    for shp in [(0, 5), (7, 0)]:
        x = torch.zeros(shp, dtype=torch.uint8, device=DEV)
        res, got = ctx.all_max_squares(x)
        assert res.cpu().tolist() == [0, -1, -1, 0] and got.shape[0] == 0
    res, got = ctx.all_max_squares(torch.zeros((50, 60), dtype=torch.uint8, device=DEV))
    assert res.cpu().tolist() == [0, -1, -1, 0] and got.shape[0] == 0


def test_state_clean_after_listing(ctx):
    """A listing call leaves the context ready: the next plain call agrees."""
    a = gen.bernoulli_u8(500, 800, 0.9, seed=31)
    a[100:180, 300:380] = 1
    check(ctx, a)
    x = torch.from_numpy(a).to(DEV)
    (K, r, c), _ = oracle.dp(a, want_map=False)
    assert ctx.max_square(x).cpu().tolist() == [K, r, c, 0]
