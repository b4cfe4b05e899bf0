"""Largest all-ones cube of 3-D volumes (bitplane growth) through the C ABI
against the oracle's 3-D recurrence: side and first corner."""
import numpy as np
import pytest

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


def check(ctx, v):
    exp = list(oracle.cube(v))
    got = ctx.max_cube(torch.from_numpy(np.ascontiguousarray(v)).to(DEV)).cpu().tolist()
    assert got[:5] == exp + [0], (v.shape, got, exp)
    return exp[0]


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 7), (7, 33, 31), (16, 64, 65),
                                   (40, 50, 100), (9, 130, 300)])
@pytest.mark.parametrize("p", [0.5, 0.9, 0.98])
def test_random_volumes(ctx, shape, p):
    rng = np.random.default_rng(hash((shape, p)) % 2**32)
    check(ctx, (rng.random(shape) < p).astype(np.uint8))


def test_planted_cubes_and_closed_forms(ctx):
    rng = np.random.default_rng(8)
    for d, m, n, s in [(40, 60, 70, 20), (70, 80, 90, 45), (64, 64, 200, 33)]:
        v = (rng.random((d, m, n)) < 0.7).astype(np.uint8)
        z, i, j = d - s - 1, (m - s) // 2, n - s
        v[z:z + s, i:i + s, j:j + s] = 1
        assert check(ctx, v) >= s
    for shp in [(5, 5, 5), (12, 40, 9), (33, 34, 35)]:
        assert check(ctx, np.ones(shp, dtype=np.uint8)) == min(shp)
        assert check(ctx, np.zeros(shp, dtype=np.uint8)) == 0
    # nonzero bytes other than 1, and a strided (sliced) view
    v = (rng.random((10, 20, 70)) < 0.9).astype(np.uint8) * rng.integers(1, 256, (10, 20, 70),
                                                                           dtype=np.uint8)
    big = torch.zeros((10, 24, 80), dtype=torch.uint8, device=DEV)
    big[:, 2:22, 5:75] = torch.from_numpy(v).to(DEV)
    exp = list(oracle.cube(v != 0))
    assert ctx.max_cube(big[:, 2:22, 5:75]).cpu().tolist()[:5] == exp + [0]


def test_empty_volumes(ctx):
    for shp in [(0, 3, 3), (3, 0, 3), (3, 3, 0)]:
        x = torch.zeros(shp, dtype=torch.uint8, device=DEV)
        assert ctx.max_cube(x).cpu().tolist()[:5] == [0, -1, -1, -1, 0]
