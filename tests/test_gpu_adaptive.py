"""Adaptive decoding (Sec. V) on the GPU against the oracle's composition:
Fast-SSC on every frame, the list decoder with L_max on CRC failures."""
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
    return torch, polar


def _check(got, ref, dtype):
    gb, gpm, gok, gsl = (t.cpu().numpy() for t in got[:4])
    ob, opm, ook, osl, _ = ref
    bad = np.flatnonzero((gb != ob).any(axis=1) | (gok != ook) | (gsl != osl))
    assert bad.size == 0, bad[:8]
    if dtype == "i8":
        assert np.array_equal(gpm, opm)
    else:
        np.testing.assert_allclose(gpm, opm, rtol=1e-5, atol=0)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("case", [(1024, 860, 3.0, 16, 600), (2048, 1723, 3.5, 32, 300)])
def test_adaptive_matches_oracle(env, oracle_mod, dtype, case):
    torch, polar = env
    N, K, snr, L, F = case
    fr = I.ga_frozen_mask(N, K, 4.0, (K - 32) / N)
    f = I.make_frames(fr, 32, I.CRC32_POLY, snr, F, seed=N + L)
    x = f.llr_i8 if dtype == "i8" else f.llr_f32
    fast = polar.PolarCode(fr, 32, I.CRC32_POLY, 1)
    lst = polar.PolarCode(fr, 32, I.CRC32_POLY, L)
    got = polar.adaptive_decode(fast, lst, torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref = oracle_mod.adaptive_decode(fr, L, x, 32, I.CRC32_POLY, n_threads=NT)
    assert 0 < ref[4] < F
    assert int(got[4].item()) == ref[4]
    _check(got, ref, dtype)
    fast.close()
    lst.close()


def test_adaptive_all_pass_and_all_fail(env, oracle_mod):
    torch, polar = env
    fr = I.ga_frozen_mask(512, 300, 2.0, 268 / 512)
    fast = polar.PolarCode(fr, 32, I.CRC32_POLY, 1)
    lst = polar.PolarCode(fr, 32, I.CRC32_POLY, 8)
    clean = I.make_frames(fr, 32, I.CRC32_POLY, 2.0, 77, seed=1, noiseless=True)
    got = polar.adaptive_decode(fast, lst, torch.from_numpy(clean.llr_f32).cuda())
    assert int(got[4].item()) == 0 and bool(got[2].all())
    noise = np.random.default_rng(2).normal(0, 1, (50, 512)).astype(np.float32)   # no codeword at all
    got = polar.adaptive_decode(fast, lst, torch.from_numpy(noise).cuda())
    ref = oracle_mod.adaptive_decode(fr, 8, noise, 32, I.CRC32_POLY, n_threads=NT)
    assert int(got[4].item()) == ref[4] >= 45
    _check(got, ref, "f32")


def test_adaptive_rejects_mismatched_codes(env):
    torch, polar = env
    fr = I.ga_frozen_mask(256, 128, 2.0, 96 / 256)
    a = polar.PolarCode(fr, 32, I.CRC32_POLY, 1)
    b = polar.PolarCode(I.ga_frozen_mask(256, 129, 2.0, 97 / 256), 32, I.CRC32_POLY, 8)
    c = polar.PolarCode(fr, 0, 0, 8)
    x = torch.zeros((4, 256), dtype=torch.float32, device="cuda")
    for fast, lst in ((a, b), (c, c)):
        with pytest.raises(polar.PolarError):
            polar.adaptive_decode(fast, lst, x)
