"""Wide lists (L = 64, 128; the paper's Fig. 3 uses L = 128): the CTA-per-frame
kernel against the oracle, element by element, with the same tolerances as
the narrow kernels."""
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


def _parity(g, o, dtype, what):
    gb, gpm, gok, gsl = (t.cpu().numpy() for t in g)
    ob, opm, ook, osl = o
    bad = np.flatnonzero((gb != ob).any(axis=1) | (gsl != osl) | (gok != ook))
    assert bad.size == 0, f"{what}: {bad.size} frames differ, first {bad[:8]}"
    if dtype == "i8":
        assert np.array_equal(gpm, opm), what
    else:
        np.testing.assert_allclose(gpm, opm, rtol=1e-5, atol=0, err_msg=what)


def _run(torch, polar, oracle_mod, fr, crc, poly, L, llr, mode=0, systematic=False):
    code = polar.PolarCode(fr, crc, poly, L, mode=mode, systematic=systematic)
    assert code.info()["warps_per_frame"][0] == L // 32
    g = code.decode(torch.from_numpy(np.ascontiguousarray(llr)).cuda())
    torch.cuda.synchronize()
    code.close()
    om = mode | (oracle_mod.SYSTEMATIC if systematic else 0)
    return g, oracle_mod.decode(fr, L, llr, crc, poly, om, n_threads=NT)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("L", [64, 128])
def test_wide_configs(env, oracle_mod, dtype, L):
    torch, polar = env
    cases = [(I.ga_frozen_mask(256, 128, 2.0, 120 / 256), 8, I.CRC8_POLY, 2.0, 120),
             (I.ga_frozen_mask(1024, 860, 4.0, 828 / 1024), 32, I.CRC32_POLY, 3.25, 40),
             (I.ga_frozen_mask(1024, 860, 4.0, 852 / 1024), 8, I.CRC8_POLY, 3.25, 40)]
    for fr, crc, poly, snr, F in cases:
        f = I.make_frames(fr, crc, poly, snr, F, seed=L + crc)
        llr = f.llr_i8 if dtype == "i8" else f.llr_f32
        g, o = _run(torch, polar, oracle_mod, fr, crc, poly, L, llr)
        _parity(g, o, dtype, f"N={fr.size} crc={crc} L={L}")


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_wide_random_codes_and_edges(env, oracle_mod, dtype, mode):
    torch, polar = env
    rng = np.random.default_rng(17 + mode)
    for N in (8, 32, 128, 256):
        K = int(rng.integers(max(2, N // 8), N))
        crc = 8 if K > 12 else 0
        fr = I.ga_frozen_mask(N, K, float(rng.uniform(0, 4)), max(K - crc, 1) / N)
        f = I.make_frames(fr, crc, I.CRC8_POLY, float(rng.uniform(-1, 3)), 16, seed=int(rng.integers(1 << 30)))
        llrs = [f.llr_f32, np.zeros((3, N), np.float32), rng.integers(-2, 3, (6, N)).astype(np.float32)]
        for x in llrs:
            llr = I.quantize_i8(x) if dtype == "i8" and x.dtype != np.int8 else x
            if dtype == "i8" and x is f.llr_f32:
                llr = f.llr_i8
            for L in (64, 128):
                g, o = _run(torch, polar, oracle_mod, fr, crc, I.CRC8_POLY, L, llr, mode)
                _parity(g, o, dtype, f"N={N} K={K} L={L} mode={mode}")


def test_wide_systematic_and_adaptive(env, oracle_mod):
    torch, polar = env
    fr = I.ga_frozen_mask(512, 300, 2.0, 268 / 512)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 1.75, 60, seed=5, systematic=True)
    g, o = _run(torch, polar, oracle_mod, fr, 32, I.CRC32_POLY, 64, f.llr_f32, systematic=True)
    _parity(g, o, "f32", "systematic L=64")
    f = I.make_frames(fr, 32, I.CRC32_POLY, 1.75, 120, seed=6)
    fast = polar.PolarCode(fr, 32, I.CRC32_POLY, 1)
    wide = polar.PolarCode(fr, 32, I.CRC32_POLY, 128)
    got = polar.adaptive_decode(fast, wide, torch.from_numpy(f.llr_i8).cuda())
    ref = oracle_mod.adaptive_decode(fr, 128, f.llr_i8, 32, I.CRC32_POLY, n_threads=NT)
    assert int(got[4].item()) == ref[4] > 0
    _parity(got[:4], ref[:4], "i8", "adaptive L_max=128")
    for name in ("set_launch",):
        with pytest.raises(polar.PolarError):
            wide.set_launch(0, 1, 0)
    fast.close()
    wide.close()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("L", [64, 128])
def test_every_shared_memory_budget(env, oracle_mod, dtype, L):
    """The wide CTA keeps its smallest buffers (low alpha stages, left betas,
    the channel row) in shared memory up to a budget and the rest in global
    scratch: from nothing on chip (budget 1) to as much as a CTA holds, with
    the scratch poisoned, the results are the oracle's."""
    torch, polar = env
    lib = polar.load_library()
    dt = polar.LLR_I8 if dtype == "i8" else polar.LLR_F32
    for N, K, crc, poly, snr in ((1024, 836, 8, I.CRC8_POLY, 3.0), (256, 128, 8, I.CRC8_POLY, 1.5),
                                 (4096, 3000, 32, I.CRC32_POLY, 3.0)):
        fr = I.ga_frozen_mask(N, K, 3.0, (K - crc) / N)
        f = I.make_frames(fr, crc, poly, snr, 24 if N == 4096 else 64, seed=N + L)
        llr = f.llr_i8 if dtype == "i8" else f.llr_f32
        o = oracle_mod.decode(fr, L, llr, crc, poly, 0, n_threads=NT)
        code = polar.PolarCode(fr, crc, poly, L)
        masks = set()
        lib.polar_debug_inject(polar.INJECT_POISON, 1)
        try:
            for budget in (1, 6000, 20000, 0, 100000, 232448):
                code.set_smem_budget(dt, budget)
                masks.add(code.info()["spill_mask"][dt])
                g = code.decode(torch.from_numpy(np.ascontiguousarray(llr)).cuda())
                torch.cuda.synchronize()
                _parity(g, o, dtype, f"N={N} L={L} budget={budget}")
        finally:
            lib.polar_debug_inject(polar.INJECT_POISON, 0)
        assert ((1 << (N.bit_length() - 1)) - 1) in masks and len(masks) >= 3
        code.close()


def test_wide_autotune_keeps_results(env, oracle_mod):
    torch, polar = env
    fr = I.ga_frozen_mask(1024, 836, 4.0, 828 / 1024)
    f = I.make_frames(fr, 8, I.CRC8_POLY, 3.0, 600, seed=8)
    llr = torch.from_numpy(f.llr_f32).cuda()
    code = polar.PolarCode(fr, 8, I.CRC8_POLY, 128)
    w, b, t = code.autotune(llr)
    assert w == 4 and t == 128 and b > 0
    g = code.decode(llr)
    torch.cuda.synchronize()
    _parity(g, oracle_mod.decode(fr, 128, f.llr_f32, 8, I.CRC8_POLY, 0, n_threads=NT), "f32", "after autotune")
    code.close()
