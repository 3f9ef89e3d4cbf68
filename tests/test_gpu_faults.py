"""Host-side fault injection and scratch poisoning (no GPU fault is ever
raised). Poisoned scratch holds bytes no decode writes (float NaN, int8
-128): a read of scratch that was never written would change the results and
fail parity. Failed allocations must come back as POLAR_ENOMEM and leave the
library usable."""
import os

import numpy as np
import pytest

from paper_1505_01466_gb300 import inputs as I

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1505_01466_gb300 import polar
    yield torch, polar
    polar.debug_inject(polar.INJECT_POISON, 0)
    polar.debug_inject(polar.INJECT_ALLOC_FAIL, -1)


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def _np(t):
    return tuple(x.cpu().numpy() for x in t)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_poisoned_scratch_changes_nothing(env, oracle_mod, dtype):
    torch, polar = env
    polar.debug_inject(polar.INJECT_POISON, 1)
    try:
        rng = np.random.default_rng(3)
        for N, L, launch in ((64, 8, (1, 0, 128)), (512, 32, (1, 7000, 512)), (512, 16, (4, 20000, 128)),
                             (2048, 32, (1, 7000, 256)), (256, 64, None)):
            K = int(rng.integers(N // 3, N - N // 8))
            fr = I.ga_frozen_mask(N, K, 3.0, (K - 32) / N)
            f = I.make_frames(fr, 32, I.CRC32_POLY, 2.5, 48, seed=N + L)
            x = f.llr_i8 if dtype == "i8" else f.llr_f32
            code = polar.PolarCode(fr, 32, I.CRC32_POLY, L)
            if launch:
                code.set_launch(1 if dtype == "i8" else 0, *launch)
            g = _np(code.decode(torch.from_numpy(x).cuda()))
            torch.cuda.synchronize()
            o = oracle_mod.decode(fr, L, x, 32, I.CRC32_POLY, 0, n_threads=NT)
            assert np.array_equal(g[0], o[0]) and np.array_equal(g[2], o[2]) and np.array_equal(g[3], o[3])
            if dtype == "i8":
                assert np.array_equal(g[1], o[1])
            else:
                np.testing.assert_allclose(g[1], o[1], rtol=1e-5, atol=0)
            code.close()
    finally:
        polar.debug_inject(polar.INJECT_POISON, 0)


def test_failed_allocations_return_enomem_and_recover(env):
    torch, polar = env
    fr = I.ga_frozen_mask(1024, 860, 4.0, 828 / 1024)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.5, 3000, seed=4)
    llr = torch.from_numpy(f.llr_f32).cuda()
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 8)
    code.set_launch(0, 1, 7000, 128)                      # a shape with global scratch
    ref = _np(code.decode(llr))
    fast = polar.PolarCode(fr, 32, I.CRC32_POLY, 1)
    try:
        polar.debug_inject(polar.INJECT_ALLOC_FAIL, 0)
        with pytest.raises(polar.PolarError) as e:
            code.decode(llr)
        assert e.value.status == polar.POLAR_ENOMEM
        # the adaptive decoder: its first decode allocates, the compaction list does not get memory
        polar.debug_inject(polar.INJECT_ALLOC_FAIL, 1)
        with pytest.raises(polar.PolarError) as e:
            polar.adaptive_decode(fast, code, llr)
        assert e.value.status == polar.POLAR_ENOMEM
        # host-buffer decode: the second staging buffer fails
        polar.debug_inject(polar.INJECT_ALLOC_FAIL, 1)
        hb = torch.empty((3000, 104), dtype=torch.uint8)
        hp = torch.empty(3000, dtype=torch.float32)
        with pytest.raises(polar.PolarError) as e:
            code.decode_host(llr.cpu(), hb, hp)
        assert e.value.status == polar.POLAR_ENOMEM
    finally:
        polar.debug_inject(polar.INJECT_ALLOC_FAIL, -1)
    torch.cuda.synchronize()
    _same(_np(code.decode(llr)), ref)                       # nothing left behind
    with pytest.raises(polar.PolarError):
        polar.debug_inject(99, 0)
    code.close()
    fast.close()
