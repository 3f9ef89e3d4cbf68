"""GPU tests of the serving form (continuous batching): each request's result
is the same alone and in the mix (and equals the plain decoder), admission
respects the device-memory budget, and waits are bounded."""
import time

import numpy as np
import pytest

from paper_1505_01466_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_01466_gb300.polar as polar
    return torch, polar


def _requests(polar, n_req, seed):
    rng = np.random.default_rng(seed)
    specs = [(256, 128, 4), (1024, 860, 8), (2048, 1723, 32), (512, 384, 16), (4096, 2048, 2)]
    codes = []
    for N, K, L in specs:
        fr = I.ga_frozen_mask(N, K, 4.0, (K - 32) / N)
        codes.append(polar.PolarCode(fr, 32, I.CRC32_POLY, L))
    reqs = []
    for r in range(n_req):
        c = int(rng.integers(len(specs)))
        n = int(np.exp(rng.uniform(0, np.log(300))))
        f = I.make_frames(codes[c].frozen, 32, I.CRC32_POLY, float(rng.uniform(3.0, 4.5)), n, seed=seed * 1000 + r)
        llr = f.llr_i8 if rng.random() < 0.5 else f.llr_f32
        reqs.append((codes[c], llr))
    return codes, reqs


def test_results_same_alone_and_in_the_mix(env):
    torch, polar = env
    codes, reqs = _requests(polar, 40, seed=7)
    srv = polar.PolarServer(device_mem_budget=256 << 20, max_frames_in_flight=1 << 16)
    alone = []
    for code, llr in reqs:
        t = srv.submit(code, llr)
        alone.append(srv.result(t))
    tickets = [srv.submit(code, llr) for code, llr in reqs]
    mixed = [srv.result(t) for t in tickets]
    st = srv.stats()
    assert st["completed"] == 2 * len(reqs)
    assert st["batches"] < 2 * len(reqs)            # requests were batched together in the mix
    # latency percentiles by request size cover the same requests
    sizes = [llr.shape[0] for _, llr in reqs]
    small, rest, every = srv.latency(1, 16), srv.latency(17, 1 << 30), srv.latency(1, 1 << 30)
    assert small["count"] == 2 * sum(1 for n in sizes if n <= 16)
    assert small["count"] + rest["count"] == every["count"] == 2 * len(reqs)
    assert every["p50_us"] == st["p50_us"] and every["p99_us"] == st["p99_us"]
    assert 0 < small["p50_us"] <= small["p99_us"] <= st["max_us"]
    with pytest.raises(polar.PolarError):
        srv.latency(5, 4)
    for (code, llr), a, m in zip(reqs, alone, mixed):
        for x, y in zip(a, m):
            assert np.array_equal(x, y)
        g = code.decode(torch.from_numpy(llr).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(a[0], g[0].cpu().numpy())
        assert np.array_equal(a[1], g[1].cpu().numpy())
        assert np.array_equal(a[2], g[2].cpu().numpy())
    srv.close()


def test_overlap_and_memory_admission(env):
    torch, polar = env
    codes, reqs = _requests(polar, 60, seed=8)
    # a budget that holds only a few requests at a time
    srv = polar.PolarServer(device_mem_budget=6 << 20, max_frames_in_flight=4096)
    big = max(r[1].nbytes for r in reqs)
    assert big < 6 << 20
    tickets = [srv.submit(code, llr) for code, llr in reqs]
    res = [srv.result(t, timeout_ms=120000) for t in tickets]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["pending"] == 0
    assert st["max_batches_in_flight"] >= 2          # batches overlapped on the device
    for (code, llr), r in zip(reqs[:10], res[:10]):
        g = code.decode(torch.from_numpy(llr).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(r[0], g[0].cpu().numpy()) and np.array_equal(r[1], g[1].cpu().numpy())
    # a request that can never fit is refused at submit
    code, llr = reqs[0]
    huge = np.zeros((8192, code.N), dtype=np.float32)
    with pytest.raises(polar.PolarError):
        srv.submit(code, huge)
    srv.close()


def test_bounded_wait_and_pause(env):
    torch, polar = env
    codes, reqs = _requests(polar, 3, seed=9)
    srv = polar.PolarServer(device_mem_budget=64 << 20, max_frames_in_flight=1 << 14, paused=True)
    t = srv.submit(*reqs[0])
    t0 = time.time()
    assert srv.wait(t, timeout_ms=50) == polar.POLAR_ETIMEDOUT
    assert time.time() - t0 < 5.0
    assert srv.poll(t) is None
    assert srv.stats()["pending"] == 1
    srv.pause(False)
    assert srv.wait(t, timeout_ms=60000) == polar.POLAR_OK
    assert srv.poll(t) is not None
    srv.close()
