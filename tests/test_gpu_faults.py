"""Failure handling, every fault made on the host (no kernel is made to fault,
trap or hang):

- a context whose workspace budget cannot hold a call's fix-up state returns
  MS_ERR_OOM, launches nothing, leaks nothing, and a later call with room is
  exact;
- a budget with room for the fix-up state but not for the bitplane scratch
  takes the strip fix-up and is still exact;
- a server batch whose launch fails (the server's test hook) completes its
  own requests with MS_ERR_CUDA while every other request is served exactly;
- a request still waiting for admission can be withdrawn: it completes with
  MS_ERR_CANCELLED, the others are unaffected; an admitted one cannot.
"""

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_18974_gb300 as m
    m.build()
    return m


def planted(m, n, s, seed, p=0.9):
    a = gen.bernoulli_u8(m, n, p, seed=seed)
    r0, c0 = (m - s) // 3, (n - s) // 2
    a[r0:r0 + s, c0:c0 + s] = 1
    return a


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_budget_too_small_returns_oom_without_leak(ms):
    """A tall matrix needs fix-up carries (16 bits per row and strip) beyond a
    300 KB budget that the context's initial workspace fits in."""
    a = planted(60000, 600, 100, seed=801)
    exp = [*oracle.freq(a), 0]
    x = torch.from_numpy(a).to(DEV)
    out = torch.full((4,), -9, dtype=torch.int32, device=DEV)
    before = free_bytes()
    for _ in range(3):  # repeated failures must not accumulate memory
        ctx = ms.MaxSquare(0, workspace_budget=300 << 10)
        with pytest.raises(ms.MSError) as e:
            ctx.max_square(x, out=out)
        assert e.value.code == 2  # MS_ERR_OOM
        ctx.close()
    after = free_bytes()
    assert abs(before - after) < (8 << 20), (before, after)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [-9, -9, -9, -9]  # nothing was launched
    ctx = ms.MaxSquare(0)
    assert ctx.max_square(x, out=out).cpu().tolist() == exp
    ctx.close()


def test_budget_without_bitplane_scratch_still_exact(ms):
    """Room for the per-matrix state and strip carries but not for the
    bitplane planes: the call takes the sequential strip fix-up."""
    a = planted(2000, 1800, 300, seed=802)
    exp = [*oracle.freq(a), 0]
    x = torch.from_numpy(a).to(DEV)
    ctx = ms.MaxSquare(0, workspace_budget=1 << 20)
    assert ctx.max_square(x).cpu().tolist() == exp
    w = torch.from_numpy(gen.pack_bits(a, a.shape[1]).view(np.int32)).to(DEV)
    assert ctx.max_square(w, n=a.shape[1]).cpu().tolist() == exp
    ctx.close()


def test_failed_batch_fails_only_its_own_requests(ms):
    mats, exps = [], []
    for k in range(3):
        a = planted(1500, 1500, 200 + 50 * k, seed=810 + k)
        mats.append(gen.pack_bits(a, 1500))
        exps.append([*oracle.freq(a), 0])
    # one request per batch at most, so the second batch is exactly request 2
    srv = ms.Server(0, memory_budget=1 << 30, streams=1, max_batch=1, test_fail_batch=2)
    ids = [srv.submit(mats[k % 3], n=1500) for k in range(6)]
    srv.wait_all()
    done = {c["id"]: c for c in srv.poll(64)}
    srv.close()
    assert len(done) == 6
    failed = [i for i in ids if done[i]["result"][3] != 0]
    assert failed == [ids[1]], [done[i]["result"] for i in ids]
    assert done[ids[1]]["result"] == [0, -1, -1, 3]  # MS_ERR_CUDA
    for k, i in enumerate(ids):
        if i != ids[1]:
            assert done[i]["result"] == exps[k % 3], (k, done[i]["result"])
    # the server's lanes recover: a new request after the failure is exact
    srv = ms.Server(0, memory_budget=1 << 30, streams=1, max_batch=4, test_fail_batch=1)
    first = srv.submit(mats[0], n=1500)
    srv.wait_all()
    second = srv.submit(mats[1], n=1500)
    srv.wait_all()
    done = {c["id"]: c for c in srv.poll(8)}
    srv.close()
    assert done[first]["result"][3] == 3
    assert done[second]["result"] == exps[1]


def test_cancel_withdraws_only_waiting_requests(ms):
    side = 4096
    a = planted(side, side, 900, seed=820)
    exp = [*oracle.freq(a), 0]
    w = gen.pack_bits(a, side)
    # the budget holds one request: the others wait for admission in order
    srv = ms.Server(0, memory_budget=w.nbytes + 4096, streams=1, max_batch=4)
    ids = [srv.submit(w, n=side) for _ in range(8)]
    cancelled = [ids[3], ids[6]]
    for i in cancelled:
        assert srv.cancel(i) == 0
    assert srv.cancel(ids[3]) == 1   # already withdrawn
    assert srv.cancel(123456789) == 1  # unknown
    srv.wait_all()
    done = {c["id"]: c for c in srv.poll(64)}
    assert srv.cancel(ids[0]) == 1   # finished long ago
    srv.close()
    assert len(done) == 8
    for i in ids:
        if i in cancelled:
            assert done[i]["result"] == [0, -1, -1, 7]  # MS_ERR_CANCELLED
        else:
            assert done[i]["result"] == exp, done[i]["result"]
