"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: an independent numpy
brute force by integral images, exhaustive enumeration of tiny matrices,
hand-derived fixtures (tests/golden), closed forms and invariants that follow
from the definition of the problem (Sec. 1, Eq. 1) and from Algorithm 1's
invariants (Sec. 3.4), and a published SplitMix64 test vector for the input
generator.
"""
import itertools
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers ---

def np_brute_batch(x: np.ndarray):
    """Independent brute force: (B, m, n) 0/1 -> arrays side, row, col.

    Uses 2-D prefix sums: the s x s window ending at (i, j) is all ones iff its
    sum is s*s.  The witness is the first (i, j) in row-major order at side K."""
    x = (np.asarray(x) != 0).astype(np.int32)
    B, m, n = x.shape
    side = np.zeros(B, dtype=np.int64)
    row = np.full(B, -1, dtype=np.int64)
    col = np.full(B, -1, dtype=np.int64)
    if m == 0 or n == 0:
        return side, row, col
    I = np.zeros((B, m + 1, n + 1), dtype=np.int32)
    I[:, 1:, 1:] = x.cumsum(1).cumsum(2)
    for s in range(1, min(m, n) + 1):
        win = I[:, s:, s:] - I[:, :-s, s:] - I[:, s:, :-s] + I[:, :-s, :-s]
        full = win == s * s  # shape (B, m-s+1, n-s+1), index (i-s+1, j-s+1)
        anyf = full.reshape(B, -1).any(1)
        if not anyf.any():
            break
        first = full.reshape(B, -1).argmax(1)
        w = n - s + 1
        side[anyf] = s
        row[anyf] = first[anyf] // w + s - 1
        col[anyf] = first[anyf] % w + s - 1
    return side, row, col


def np_brute(a):
    s, r, c = np_brute_batch(np.asarray(a)[None])
    return int(s[0]), int(r[0]), int(c[0])


def heights(a):
    a = np.asarray(a) != 0
    h = np.zeros(a.shape, dtype=np.int64)
    for i in range(a.shape[0]):
        h[i] = np.where(a[i], (h[i - 1] + 1) if i else 1, 0)
    return h


def load_golden(path):
    mat, dpm, expect, mode = [], [], None, "mat"
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("expect"):
                expect = tuple(int(t) for t in line.split()[1:4])
                continue
            if line == "dp":
                mode = "dp"
                continue
            (mat if mode == "mat" else dpm).append([int(t) for t in line.split()])
    return (np.array(mat, dtype=np.uint8), expect,
            np.array(dpm, dtype=np.int32) if dpm else None)


ALL_SIDES = ("dp", "dp_rows", "freq", "freq_dpmap", "brute")


def all_oracles(a):
    return {
        "dp": oracle.dp(a, want_map=False)[0],
        "dp_rows": oracle.dp_rows(a),
        "freq": oracle.freq(a),
        "freq_dpmap": oracle.freq_dpmap(a)[0],
        "brute": oracle.brute(a),
    }


# ---------------------------------------------------------------- generator -

def test_splitmix64_published_vector():
    # SplitMix64 started from state 0 (Steele, Lea & Flood 2014; the reference
    # seeding routine of the xoshiro generators) outputs these two values first.
    gamma = 0x9E3779B97F4A7C15
    assert gen.mix64(gamma) == 0xE220A8397B1DCDAF
    assert gen.mix64((2 * gamma) & (2**64 - 1)) == 0x6E789E6AA1B965F4


def test_generator_counter_form_and_density():
    # draw(seed, k) is output k of a SplitMix64 stream whose state starts at mix(seed)
    key = gen.mix64(7)
    gamma = 0x9E3779B97F4A7C15
    for k in range(5):
        assert gen.draw(7, k) == gen.mix64((key + (k + 1) * gamma) & (2**64 - 1))
    a = gen.bernoulli_u8(300, 400, 0.3, seed=11)
    # cell (i,j) is draw(i*n+j) >> 40 < thr24
    thr = gen.thr24(0.3)
    for (i, j) in [(0, 0), (5, 7), (299, 399), (123, 45)]:
        assert a[i, j] == int((gen.draw(11, i * 400 + j) >> 40) < thr)
    assert abs(a.mean() - 0.3) < 0.01
    assert set(np.unique(a)) <= {0, 1}
    assert gen.thr24(0.0) == 0 and gen.thr24(1.0) == 1 << 24
    assert gen.bernoulli_u8(10, 10, 1.0, 3).all()
    assert not gen.bernoulli_u8(10, 10, 0.0, 3).any()


def test_generator_ld_and_plant():
    a = gen.bernoulli_u8(50, 60, 0.5, seed=3, ld=64)
    b = gen.bernoulli_u8(50, 60, 0.5, seed=3)
    assert np.array_equal(a[:, :60], b)
    assert not a[:, 60:].any()
    for (m, n, s) in [(100, 80, 10), (600, 601, 600), (32, 32, 1)]:
        r, c = gen.plant_pos(5, m, n, s)
        assert 0 <= r <= m - s and 0 <= c <= n - s


def test_pack_roundtrip_and_padding():
    a = gen.bernoulli_u8(37, 70, 0.5, seed=9)
    for pad in (0, 1):
        w = gen.pack_bits(a, 70, ldw=4, pad_value=pad)
        assert w.shape == (37, 4)
        assert np.array_equal(oracle.unpack(w, 37, 70), a)
        assert np.array_equal(gen.unpack_bits(w, 37, 70), a)
    # bit b of word w is column 32*w+b
    z = np.zeros((1, 40), dtype=np.uint8)
    z[0, 33] = 1
    w = gen.pack_bits(z, 40)
    assert w[0, 0] == 0 and w[0, 1] == 2


# ---------------------------------------------------------------- pins ------

@pytest.mark.parametrize("name", sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt")))
def test_golden(name):
    a, expect, dpm = load_golden(os.path.join(GOLDEN, name))
    for k, v in all_oracles(a).items():
        assert v == expect, (k, v, expect)
    assert np_brute(a) == expect
    if dpm is not None:
        assert np.array_equal(oracle.dp(a)[1], dpm)
        assert np.array_equal(oracle.freq_dpmap(a)[1], dpm)


def _shapes(maxcells):
    for m in range(1, maxcells + 1):
        for n in range(1, maxcells // m + 1):
            yield m, n


def test_exhaustive_tiny():
    """Every 0/1 matrix with m*n <= 12 cells, plus every 4x4 matrix."""
    shapes = list(_shapes(12)) + [(4, 4)]
    for (m, n) in shapes:
        cells = m * n
        codes = np.arange(1 << cells, dtype=np.int64)
        X = ((codes[:, None] >> np.arange(cells)) & 1).astype(np.uint8).reshape(-1, m, n)
        side, row, col = np_brute_batch(X)
        for b in range(X.shape[0]):
            exp = (int(side[b]), int(row[b]), int(col[b]))
            a = X[b]
            assert oracle.dp(a, want_map=False)[0] == exp, (m, n, b)
            assert oracle.freq(a) == exp, (m, n, b)
            if cells <= 9 or b % 7 == 0:
                assert oracle.freq_dpmap(a)[0] == exp
                assert oracle.brute(a) == exp
                assert oracle.dp_rows(a) == exp


def test_random_small_against_brute():
    rng = np.random.default_rng(1234)
    for t in range(1500):
        m, n = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        p = float(rng.choice([0.1, 0.3, 0.5, 0.7, 0.8, 0.9, 0.95]))
        a = (rng.random((m, n)) < p).astype(np.uint8)
        exp = np_brute(a)
        got = all_oracles(a)
        for k, v in got.items():
            assert v == exp, (k, v, exp, a)
        assert np.array_equal(oracle.dp(a)[1], oracle.freq_dpmap(a)[1])


def test_closed_forms():
    for (m, n) in [(1, 1), (1, 9), (9, 1), (5, 5), (7, 3), (64, 100), (130, 129)]:
        ones = np.ones((m, n), dtype=np.uint8)
        s = min(m, n)
        for k, v in all_oracles(ones).items():
            assert v == (s, s - 1, s - 1), k
        ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
        assert np.array_equal(oracle.dp(ones)[1], np.minimum(ii, jj) + 1)
        zeros = np.zeros((m, n), dtype=np.uint8)
        for k, v in all_oracles(zeros).items():
            assert v == (0, -1, -1), k
        assert not oracle.dp(zeros)[1].any()
    # a single one
    for (m, n, i, j) in [(1, 1, 0, 0), (8, 9, 3, 4), (20, 3, 19, 2)]:
        a = np.zeros((m, n), dtype=np.uint8)
        a[i, j] = 1
        for k, v in all_oracles(a).items():
            assert v == (1, i, j), k
    # checkerboards: side 1, first one in row-major order
    for (m, n, phase) in [(4, 4, 0), (5, 6, 1), (33, 31, 0)]:
        ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
        a = ((ii + jj + phase) % 2 == 0).astype(np.uint8)
        exp = (1, 0, 0) if phase == 0 else (1, 0, 1)
        for k, v in all_oracles(a).items():
            assert v == exp, k
    # 1 x n: side 1 iff any one, witness at the first one
    a = np.zeros((1, 10), dtype=np.uint8)
    a[0, [4, 7]] = 1
    for k, v in all_oracles(a).items():
        assert v == (1, 0, 4)
    # empty matrices (Algorithm 1 returns 0 for an empty input)
    for shp in [(0, 5), (5, 0), (0, 0)]:
        e = np.zeros(shp, dtype=np.uint8)
        for k, v in all_oracles(e).items():
            assert v == (0, -1, -1), k
    # any nonzero byte is a one
    a = np.array([[3, 255], [17, 1]], dtype=np.uint8)
    for k, v in all_oracles(a).items():
        assert v == (2, 1, 1)


def test_invariants_random():
    rng = np.random.default_rng(77)
    for t in range(40):
        m, n = int(rng.integers(20, 120)), int(rng.integers(20, 120))
        p = float(rng.choice([0.5, 0.7, 0.9, 0.97]))
        a = (rng.random((m, n)) < p).astype(np.uint8)
        (K, r, c), d = oracle.dp(a)
        # oracles agree, maps agree
        assert oracle.freq(a) == (K, r, c)
        assert oracle.dp_rows(a) == (K, r, c)
        (K2, _, _), d2 = oracle.freq_dpmap(a)
        assert np.array_equal(d, d2)
        # witness = first row-major argmax of the map
        flat = int(np.argmax(d.reshape(-1)))
        assert (K, r, c) == ((int(d.max()), flat // n, flat % n) if K else (0, -1, -1))
        # transpose invariance of the side
        assert oracle.dp(a.T.copy(), want_map=False)[0][0] == K
        # dp <= vertical run, horizontal run, min(i, j)+1
        h = heights(a)
        left = heights(a.T.copy()).T
        ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
        assert (d <= h).all() and (d <= left).all() and (d <= np.minimum(ii, jj) + 1).all()
        # S(i) <= S(i-1) + 1 (largest square with bottom row <= i)
        S = np.maximum.accumulate(d.max(1))
        assert (np.diff(S) <= 1).all()
        # turning a zero into a one never lowers the side
        zs = np.argwhere(a == 0)
        if len(zs):
            b = a.copy()
            b[tuple(zs[rng.integers(len(zs))])] = 1
            assert oracle.dp(b, want_map=False)[0][0] >= K
        # a planted square is a lower bound
        s = int(rng.integers(1, min(m, n) + 1))
        b = a.copy()
        i0, j0 = int(rng.integers(0, m - s + 1)), int(rng.integers(0, n - s + 1))
        b[i0:i0 + s, j0:j0 + s] = 1
        assert oracle.freq(b)[0] >= s


def test_erode_definition_and_composition():
    """S_t from oracle_erode equals [dp >= t]; and the bitplane growth identity
    S_{a+b-1}(i,j) = S_a(i,j) & S_a(i-b+1,j) & S_a(i,j-b+1) & S_a(i-b+1,j-b+1)
    for 1 <= b <= a+1 (out-of-range reads as 0) holds on random inputs."""
    rng = np.random.default_rng(5)
    for t in range(12):
        m, n = int(rng.integers(10, 60)), int(rng.integers(10, 60))
        a = (rng.random((m, n)) < 0.85).astype(np.uint8)
        a[3:3 + 9, 4:4 + 9] = 1
        _, d = oracle.dp(a)
        S = {s: oracle.erode(a, s) for s in range(1, 14)}
        for s, e in S.items():
            assert np.array_equal(e, (d >= s).astype(np.uint8)), s

        def sh(x, di, dj):
            y = np.zeros_like(x)
            y[di:, dj:] = x[:m - di, :n - dj]
            return y

        for A in range(1, 7):
            for b in range(1, A + 2):
                comp = S[A] & sh(S[A], b - 1, 0) & sh(S[A], 0, b - 1) & sh(S[A], b - 1, b - 1)
                assert np.array_equal(comp, S[A + b - 1]), (A, b)


def test_generated_config_shapes_small():
    """The 256x256, p=0.5, seed 0 workload: all oracles agree (no stored value)."""
    a = gen.bernoulli_u8(256, 256, 0.5, seed=0)
    res = all_oracles(a)
    assert len(set(res.values())) == 1
    (K, r, c) = res["dp"]
    assert 3 <= K <= 10 and r >= 0 and c >= 0


# ------------------------------------------------------ all maximal squares -

def np_all_max(a):
    """Independent enumeration: K by integral images, then every top-left
    (r, c) whose K x K window sums to K*K, reported as its bottom-right corner
    (r + K - 1, c + K - 1), sorted row-major."""
    x = (np.asarray(a) != 0).astype(np.int64)
    m, n = x.shape
    K = np_brute(x)[0]
    if K == 0:
        return 0, []
    I = np.zeros((m + 1, n + 1), dtype=np.int64)
    I[1:, 1:] = x.cumsum(0).cumsum(1)
    win = I[K:, K:] - I[:-K, K:] - I[K:, :-K] + I[:-K, :-K]
    rs, cs = np.nonzero(win == K * K)
    return K, sorted((int(r) + K - 1, int(c) + K - 1) for r, c in zip(rs, cs))


def test_all_max_against_enumeration():
    rng = np.random.default_rng(77)
    for trial in range(400):
        m, n = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        a = (rng.random((m, n)) < rng.uniform(0.3, 0.95)).astype(np.uint8)
        (K, r, c), corners = oracle.all_max(a)
        K2, want = np_all_max(a)
        assert K == K2
        assert [tuple(p) for p in corners.tolist()] == want  # row-major order
        if K:
            assert (r, c) == want[0]
    # every 3 x 3 matrix
    for bits in range(1 << 9):
        a = np.array([(bits >> k) & 1 for k in range(9)], dtype=np.uint8).reshape(3, 3)
        K, want = np_all_max(a)
        assert [tuple(p) for p in oracle.all_max(a)[1].tolist()] == want


def test_all_max_closed_forms():
    # all ones, m >= n: the n-squares stacked down the only column band
    for m, n in [(1, 1), (5, 5), (9, 4), (4, 9), (30, 7)]:
        (K, _, _), corners = oracle.all_max(np.ones((m, n), dtype=np.uint8))
        s = min(m, n)
        assert K == s
        want = [(i, j) for i in range(s - 1, m) for j in range(s - 1, n)]
        assert [tuple(p) for p in corners.tolist()] == want
        assert len(want) == (m - s + 1) * (n - s + 1)
    # all zeros and empty: no square at all
    assert oracle.all_max(np.zeros((6, 7), dtype=np.uint8))[1].shape == (0, 2)
    assert oracle.all_max(np.zeros((0, 7), dtype=np.uint8))[1].shape == (0, 2)
    # two disjoint planted squares of the same largest side in a sparse field
    a = np.zeros((40, 50), dtype=np.uint8)
    a[3:11, 5:13] = 1
    a[20:28, 30:38] = 1
    (K, r, c), corners = oracle.all_max(a)
    assert K == 8 and [tuple(p) for p in corners.tolist()] == [(10, 12), (27, 37)]
    assert (r, c) == (10, 12)


# ------------------------------------------------------------- 3-D cubes ----

def np_cube(v):
    """Independent enumeration: 3-D prefix sums; the t-cube ending at
    (z, i, j) is all ones iff its sum is t^3; the first corner in (z, i, j)
    order at the largest t."""
    x = (np.asarray(v) != 0).astype(np.int64)
    d, m, n = x.shape
    if x.size == 0:
        return (0, -1, -1, -1)
    S = np.zeros((d + 1, m + 1, n + 1), dtype=np.int64)
    S[1:, 1:, 1:] = x.cumsum(0).cumsum(1).cumsum(2)
    best = (0, -1, -1, -1)
    for t in range(1, min(d, m, n) + 1):
        w = (S[t:, t:, t:] - S[:-t, t:, t:] - S[t:, :-t, t:] - S[t:, t:, :-t]
             + S[:-t, :-t, t:] + S[:-t, t:, :-t] + S[t:, :-t, :-t] - S[:-t, :-t, :-t])
        hit = np.argwhere(w == t ** 3)
        if len(hit) == 0:
            break
        z, i, j = hit[0]  # argwhere is in (z, i, j) lexicographic order
        best = (t, int(z) + t - 1, int(i) + t - 1, int(j) + t - 1)
    return best


def test_cube_against_enumeration():
    rng = np.random.default_rng(2025)
    for trial in range(300):
        d, m, n = (int(rng.integers(1, 8)) for _ in range(3))
        v = (rng.random((d, m, n)) < rng.uniform(0.5, 0.97)).astype(np.uint8)
        assert oracle.cube(v) == np_cube(v), (d, m, n)
    # every 2 x 2 x 2 volume
    for bits in range(256):
        v = np.array([(bits >> k) & 1 for k in range(8)], dtype=np.uint8).reshape(2, 2, 2)
        assert oracle.cube(v) == np_cube(v)


def test_cube_closed_forms_and_slices():
    for d, m, n in [(1, 1, 1), (3, 5, 7), (6, 4, 9), (8, 8, 8)]:
        s = min(d, m, n)
        assert oracle.cube(np.ones((d, m, n), dtype=np.uint8)) == (s, s - 1, s - 1, s - 1)
        assert oracle.cube(np.zeros((d, m, n), dtype=np.uint8)) == (0, -1, -1, -1)
    assert oracle.cube(np.zeros((0, 3, 3), dtype=np.uint8)) == (0, -1, -1, -1)
    # one slice: a cube of side 1 at most, the first one in the slice
    rng = np.random.default_rng(4)
    a = (rng.random((20, 30)) < 0.6).astype(np.uint8)
    first = np.argwhere(a)[0]
    assert oracle.cube(a[None]) == (1, 0, int(first[0]), int(first[1]))
    # a planted cube in a sparse volume, and a stack of planted squares of
    # side s over s slices is a cube
    v = np.zeros((12, 15, 16), dtype=np.uint8)
    v[2:7, 4:9, 3:8] = 1
    assert oracle.cube(v) == (5, 6, 8, 7)
    v2 = (rng.random((10, 40, 40)) < 0.3).astype(np.uint8)
    v2[1:7, 10:16, 20:26] = 1
    assert oracle.cube(v2)[0] == 6
