"""ms_max_square_noalloc, the entry point for callers that may not allocate
device memory (for example plug-ins whose host application owns all device
memory through its own pool, or services that must not allocate after
start-up): called through the C ABI, it must give exactly the result of
ms_max_square on the same inputs, and the oracle's (the textbook DP of Eq. 1:
side and first row-major corner), on consecutive calls that reuse its fixed
scratch array, up to its largest accepted size (8192 x 8192).  This file is
named to be collected last."""
import ctypes

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_18974_gb300 as ms
    ms.build()
    L = ms.lib()
    L.ms_max_square_noalloc.restype = ctypes.c_int
    L.ms_max_square_noalloc.argtypes = [ctypes.POINTER(ms._Matrix), ctypes.c_void_p,
                                        ctypes.c_void_p]
    ctx = ms.MaxSquare(0)
    yield ms, L, ctx
    ctx.close()


def noalloc(ms, L, x, n=None, fmt=None):
    desc = ms.describe(x, n, fmt)
    out = torch.full((4,), -9, dtype=torch.int32, device=x.device)
    stream = torch.cuda.current_stream().cuda_stream or None
    rc = L.ms_max_square_noalloc(ctypes.byref(desc), out.data_ptr(), stream)
    return rc, out


def cases():
    # the second matrix of each pair has a smaller answer than the first, so a
    # result left over in the shared scratch would show
    a = gen.bernoulli_u8(700, 1500, 0.9, seed=71)
    a[100:300, 400:600] = 1            # side 200: flagged tiles, strip carries used
    b = gen.bernoulli_u8(650, 900, 0.5, seed=72)
    c = gen.bernoulli_u8(8192, 8192, 0.85, seed=73)   # the largest accepted size
    c[5000:5400, 7000:7400] = 1
    return [a, b, c, b]


def test_noalloc_matches_ms_max_square_on_consecutive_calls(libs):
    ms, L, ctx = libs
    for a in cases():
        exp = [*oracle.dp(a, want_map=False)[0], 0]
        x = torch.from_numpy(a).to("cuda:0")
        ref = ctx.max_square(x)
        rc, got = noalloc(ms, L, x)
        assert rc == 0
        assert got.cpu().tolist() == ref.cpu().tolist() == exp
        n = a.shape[1]
        w = torch.from_numpy(gen.pack_bits(a, n, pad_value=1).view(np.int32)).to("cuda:0")
        ref_b = ctx.max_square(w, n=n)
        rc, got_b = noalloc(ms, L, w, n=n)
        assert rc == 0
        assert got_b.cpu().tolist() == ref_b.cpu().tolist() == ref.cpu().tolist()


def test_noalloc_rejects_sizes_beyond_its_scratch(libs):
    ms, L, ctx = libs
    for shape in [(8193, 16), (16, 8193)]:
        x = torch.zeros(shape, dtype=torch.uint8, device="cuda:0")
        rc, out = noalloc(ms, L, x)
        assert rc == 6  # MS_ERR_UNSUPPORTED, nothing launched
        assert out.cpu().tolist() == [-9, -9, -9, -9]
    x = torch.zeros((0, 5), dtype=torch.uint8, device="cuda:0")
    rc, out = noalloc(ms, L, x)
    assert rc == 0 and out.cpu().tolist() == [0, -1, -1, 0]
