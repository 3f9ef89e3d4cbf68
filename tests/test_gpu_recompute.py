"""Stages evaluated from the channel (polar_code_set_recompute) on the GPU.

The top alpha stages of a code may be left unstored: an F or G that reads one
evaluates it from the channel row and the paths' left-sibling betas by
Eqs. (1)-(2). Results must not depend on how many stages are evaluated that
way, under every launch shape, and must equal the oracle's.
"""
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
    import oracle
    oracle.build()
    from paper_1505_01466_gb300 import polar
    return torch, polar, oracle


def _decode(torch, code, llr):
    bits, pm, ok, slot = code.decode(llr)
    torch.cuda.synchronize()
    return bits.cpu().numpy(), pm.cpu().numpy(), ok.cpu().numpy(), slot.cpu().numpy()


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_headline_code_every_depth_and_shape(env, dtype):
    torch, polar, oracle = env
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.5, 640, seed=901)
    x = f.llr_i8 if dtype == "i8" else f.llr_f32
    dt = polar.LLR_I8 if dtype == "i8" else polar.LLR_F32
    llr = torch.from_numpy(x).cuda()
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 32)
    info = code.info()
    assert info["max_recompute_depth"] == 2          # stage 8 holds a Rate-1 leaf of 256 bits
    want = oracle.decode(fr, 32, x[:96], 32, I.CRC32_POLY, oracle.SPC4, n_threads=NT)
    ref = None
    for shape in ((1, 7000, 512), (1, 16000, 256), (2, 20000, 256), (4, 60000, 128)):
        code.set_launch(dt, *shape)
        for depth in (0, 1, 2):
            code.set_recompute(dt, depth)
            mask = code.info()["recomputed_stages"][dt]
            assert mask == (((1 << depth) - 1) << (11 - depth) if depth else 0)
            got = _decode(torch, code, llr)
            if ref is None:
                ref = got
                g = tuple(v[:96] for v in got)
                assert np.array_equal(g[0], want[0]) and np.array_equal(g[3], want[3])
                assert np.array_equal(g[2], want[2])
                if dtype == "i8":
                    assert np.array_equal(g[1], want[1])
                else:
                    np.testing.assert_allclose(g[1], want[1], rtol=1e-5, atol=0)
            assert _same(got, ref), (shape, depth)
    with pytest.raises(polar.PolarError):
        code.set_recompute(dt, 3)
    code.close()


def _random_code_with_inner_top(rng, N, K):
    """A random frozen set whose top stages hold only inner nodes: each half
    and quarter of the code has both frozen and information bits away from
    the leaf patterns (not all frozen, not all information, not a
    repetition or SPC pattern)."""
    while True:
        fr = np.ones(N, np.uint8)
        fr[rng.choice(N, K, replace=False)] = 0
        ok = True
        for parts in (2, 4, 8):
            for q in np.split(fr, parts):
                nf = int(q.sum())
                rep = nf == q.size - 1 and q[-1] == 0
                spc = nf == 1 and q[0] == 1
                if nf in (0, q.size) or rep or spc:
                    ok = False
        if ok:
            return fr


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_random_codes_all_depths_equal_the_oracle(env, dtype, mode):
    torch, polar, oracle = env
    rng = np.random.default_rng(77 + mode)
    for N, L in ((512, 4), (1024, 8), (2048, 16), (4096, 32), (1024, 32), (512, 2)):
        K = int(rng.integers(N // 4, 3 * N // 4))
        fr = _random_code_with_inner_top(rng, N, K)
        crc = 8
        f = I.make_frames(fr, crc, I.CRC8_POLY, float(rng.uniform(0.5, 2.5)), 400, seed=int(rng.integers(1 << 30)))
        x = f.llr_i8 if dtype == "i8" else f.llr_f32
        dt = polar.LLR_I8 if dtype == "i8" else polar.LLR_F32
        llr = torch.from_numpy(x).cuda()
        code = polar.PolarCode(fr, crc, I.CRC8_POLY, L, mode=mode)
        vmax = code.info()["max_recompute_depth"]
        assert vmax == 3                                  # stages n-1 .. n-3 hold inner nodes only
        code.set_launch(dt, 1, 0, 256)
        outs = []
        for depth in range(vmax + 1):
            code.set_recompute(dt, depth)
            outs.append(_decode(torch, code, llr))
        for o in outs[1:]:
            assert _same(o, outs[0]), (N, L)
        want = oracle.decode(fr, L, x[:40], crc, I.CRC8_POLY, mode, n_threads=NT)
        g = tuple(v[:40] for v in outs[-1])
        assert np.array_equal(g[0], want[0]) and np.array_equal(g[3], want[3]) and np.array_equal(g[2], want[2])
        if dtype == "i8":
            assert np.array_equal(g[1], want[1])
        else:
            np.testing.assert_allclose(g[1], want[1], rtol=1e-5, atol=0)
        code.close()


def test_recompute_with_poisoned_scratch(env):
    """Scratch filled with NaN before every decode: a stage that is evaluated
    never reads the scratch, so the results stay those of the oracle."""
    torch, polar, oracle = env
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.75, 400, seed=17)
    llr = torch.from_numpy(f.llr_f32).cuda()
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 32)
    code.set_launch(polar.LLR_F32, 1, 7000, 512)
    code.set_recompute(polar.LLR_F32, 2)
    lib = polar.load_library()
    lib.polar_debug_inject(polar.INJECT_POISON, 1)
    try:
        got = _decode(torch, code, llr)
    finally:
        lib.polar_debug_inject(polar.INJECT_POISON, 0)
    want = oracle.decode(fr, 32, f.llr_f32[:64], 32, I.CRC32_POLY, oracle.SPC4, n_threads=NT)
    assert np.array_equal(got[0][:64], want[0]) and np.array_equal(got[3][:64], want[3])
    code.close()
