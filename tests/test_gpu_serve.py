"""The request server: admission by device-memory budget, resident buffers and
continuous batching.  Every result must equal ms_max_square on the same
matrix alone (bit for bit), the arena must never exceed the budget, and
requests submitted while batches run must join later, overlapping batches."""
import time

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


def make_requests(count, seed, max_side=900):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        m = int(np.exp(rng.uniform(np.log(8), np.log(max_side))))
        n = int(np.exp(rng.uniform(np.log(8), np.log(max_side))))
        a = gen.bernoulli_u8(m, n, float(rng.uniform(0.1, 0.95)), seed=seed * 1000 + i)
        if i % 3 == 0:
            s = int(rng.integers(1, min(m, n) + 1))
            a[m - s:, :s] = 1
        if i % 2:
            reqs.append((gen.pack_bits(a, n, pad_value=1), n, 1, a))
        else:
            reqs.append((np.ascontiguousarray(a), n, 0, a))
    return reqs


def test_serve_results_equal_standalone_and_budget_holds(ms):
    reqs = make_requests(80, seed=5)
    budget = 2 << 20  # small: admission has to wait for buffers to free up
    srv = ms.Server(0, memory_budget=budget, streams=2, max_batch=16)
    ids = {}
    for k, (payload, n, fmt, a) in enumerate(reqs):
        ids[srv.submit(payload, n=n, fmt=fmt)] = k
    srv.wait_all()
    done = srv.poll(1000)
    stats = srv.stats()
    srv.close()
    assert len(done) == len(reqs)
    assert stats["completed"] == stats["submitted"] == len(reqs)
    assert 0 < stats["peak_bytes"] <= budget
    ctx = ms.MaxSquare(0)
    for c in done:
        payload, n, fmt, a = reqs[ids[c["id"]]]
        if fmt == 0:
            alone = ctx.max_square(torch.from_numpy(payload).cuda())
        else:
            alone = ctx.max_square(torch.from_numpy(payload.view(np.int32)).cuda(), n=n)
        assert c["result"] == alone.cpu().tolist()
        assert c["result"][:3] == list(oracle.dp(a, want_map=False)[0])
        assert c["t_submit"] <= c["t_admit"] <= c["t_launch"] <= c["t_done"]
    ctx.close()


def test_serve_refuses_requests_that_can_never_fit(ms):
    srv = ms.Server(0, memory_budget=1 << 20, streams=1, max_batch=4)
    big = np.ones((2048, 2048), dtype=np.uint8)
    with pytest.raises(ms.MSError) as e:
        srv.submit(big)
    assert e.value.code == 5  # MS_ERR_BUDGET
    small = np.ones((64, 64), dtype=np.uint8)
    srv.submit(small)
    srv.wait_all()
    assert srv.poll()[0]["result"] == [64, 63, 63, 0]
    srv.close()


def test_serve_continuous_batching_overlaps(ms):
    """A second wave submitted while the first wave's batch is on the device
    is batched separately and runs on another stream, overlapping it."""
    srv = ms.Server(0, memory_budget=1 << 30, streams=2, max_batch=64)
    wave, exp = [], []
    for i in range(2):
        a = gen.bernoulli_u8(8192, 8192, 0.9, seed=40 + i)
        a[1000:4000, 500:3500] = 1  # a large square: the exact fix-up runs for a while
        wave.append(gen.pack_bits(a, 8192))
        exp.append([*oracle.freq(a), 0])
    first = [srv.submit(wave[k % 2], n=8192) for k in range(12)]
    t0 = time.time()
    while srv.stats()["batches"] < 1 and time.time() - t0 < 10:
        time.sleep(0.0002)
    second = [srv.submit(wave[1], n=8192) for _ in range(4)]
    srv.wait_all()
    done = {c["id"]: c for c in srv.poll(100)}
    stats = srv.stats()
    srv.close()
    assert stats["batches"] >= 2
    assert exp[0][0] >= 3000 and exp[1][0] >= 3000
    for k, i in enumerate(first):
        assert done[i]["result"] == exp[k % 2], (k, done[i]["result"], exp[k % 2])
    for i in second:
        assert done[i]["result"] == exp[1]
    t_done_first = min(done[i]["t_done"] for i in first)
    assert any(done[i]["t_launch"] < t_done_first for i in second) or stats["peak_inflight"] >= 2
