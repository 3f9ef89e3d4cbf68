"""Register subtrees of lists with L <= 16 paths.

With packing on, such a frame's selection (Algorithm 1) sorts, scans and
reduces inside an L-lane segment of its warp, and rounds where every frame
group of a CTA holds a frame run the subtrees 32 / L frames to a warp (lane
f * L + s is path s of frame f). With it off a frame has its own warp and
selects over all 32 lanes. The results must be the oracle's for every list
size, node set, LLR type and CTA size, packed or not, including rounds that
are not full (a frame count that is not a multiple of the CTA's frames), in
the plain and in the batched form (classes that pack beside classes that do
not, in one launch).
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


def _check(g, o, dtype, what):
    gb, gpm, gok, gsl = (t.cpu().numpy() for t in g)
    ob, opm, ook, osl = o
    bad = np.flatnonzero((gb != ob).any(axis=1) | (gsl != osl) | (gok != ook))
    assert bad.size == 0, f"{what}: {bad.size} frames differ, first {bad[:8]}"
    if dtype == "i8":
        assert np.array_equal(gpm, opm), what
    else:
        np.testing.assert_allclose(gpm, opm, rtol=1e-5, atol=0, err_msg=what)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("L", [1, 2, 4, 8, 16])
def test_packed_subtrees_equal_the_oracle(env, dtype, L):
    torch, polar, oracle = env
    rng = np.random.default_rng(100 + L)
    dt = polar.LLR_I8 if dtype == "i8" else polar.LLR_F32
    for mode in (0, 1, 2):
        for N in (64, 256, 1024):
            K = int(rng.integers(N // 4, N - N // 8))
            crc = 8
            fr = I.ga_frozen_mask(N, K, float(rng.uniform(0.5, 3.0)), (K - crc) / N)
            F = 1000 + int(rng.integers(0, 37))                 # not a multiple of any CTA's frames
            f = I.make_frames(fr, crc, I.CRC8_POLY, float(rng.uniform(0.0, 2.5)), F, seed=int(rng.integers(1 << 30)))
            llr = f.llr_i8 if dtype == "i8" else f.llr_f32
            if dtype == "i8":
                llr[:16] = rng.integers(-3, 4, (16, N))          # ties
            o = oracle.decode(fr, L, llr, crc, I.CRC8_POLY, mode, n_threads=NT)
            x = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
            # a small batch of a fresh code runs the latency shape
            code = polar.PolarCode(fr, crc, I.CRC8_POLY, L, mode=mode)
            g = code.decode(x[:100])
            torch.cuda.synchronize()
            _check(g, tuple(t[:100] for t in o), dtype, f"latency shape L={L} N={N} mode={mode}")
            for cta in (32, 128, 256, 512):
                code.set_launch(dt, 1, 0, cta)
                for on in (False, True):
                    # on: 32 / L frames to a warp where the CTA has that many frame
                    # groups, segments alone elsewhere; off: lane-per-path selection
                    # over the whole warp
                    code.set_packing(dt, on)
                    assert code.info()["packed"][dt] == int(on)
                    g = code.decode(x)
                    torch.cuda.synchronize()
                    _check(g, o, dtype, f"packed={on} L={L} N={N} mode={mode} cta={cta}")
            code.close()


def test_packed_subtrees_in_the_batched_form(env):
    """A mix of L = 2..16 classes (and one L = 32) in one persistent launch
    with 512-thread CTAs: L = 2, 4 pack by default, one L = 8 class and the
    L = 16 class are told to, the other L = 8 class is not."""
    torch, polar, oracle = env
    rng = np.random.default_rng(7)
    classes = [(256, 128, 2), (256, 160, 4), (512, 300, 8), (1024, 700, 16), (256, 200, 32), (128, 64, 8)]
    codes, frozen, llrs = [], [], []
    for N, K, L in classes:
        fr = I.ga_frozen_mask(N, K, 2.0, (K - 32) / N)
        frozen.append(fr)
        code = polar.PolarCode(fr, 32, I.CRC32_POLY, L)
        if (N, L) in ((512, 8), (1024, 16)):
            code.set_launch(polar.LLR_I8, 1, 7000, 512)
            code.set_packing(polar.LLR_I8, True)
        codes.append(code)
        llrs.append(I.make_frames(fr, 32, I.CRC32_POLY, 2.0, 700, seed=N + L).llr_i8)
    fc = np.repeat(np.arange(len(classes), dtype=np.uint32), 700)
    rng.shuffle(fc)
    plan = polar.PolarBatch(codes, fc, polar.LLR_I8)
    llr_bytes, bits_bytes, lo, bo = plan.layout()
    packed = np.zeros(llr_bytes, np.int8)
    seen = [0] * len(classes)
    for i, c in enumerate(fc):
        N = classes[c][0]
        packed[lo[i]: lo[i] + N] = llrs[c][seen[c]]
        seen[c] += 1
    bits = torch.zeros(bits_bytes, dtype=torch.uint8, device="cuda")
    pm = torch.zeros(fc.size, dtype=torch.float32, device="cuda")
    ok = torch.zeros(fc.size, dtype=torch.uint8, device="cuda")
    plan.set_launch(1, 7000, 512)
    plan.run(torch.from_numpy(packed).cuda(), bits, pm, ok)
    torch.cuda.synchronize()
    pm = pm.cpu().numpy()
    bits = bits.cpu().numpy()
    ok = ok.cpu().numpy()
    for c, (N, K, L) in enumerate(classes):
        sel = np.flatnonzero(fc == c)
        ob, opm, ook, _ = oracle.decode(frozen[c], L, llrs[c], 32, I.CRC32_POLY, 0, n_threads=NT)
        kb = (K - 32 + 7) // 8
        got_bits = np.stack([bits[bo[i]: bo[i] + kb] for i in sel])
        assert np.array_equal(got_bits, ob), (N, K, L)
        assert np.array_equal(pm[sel], opm) and np.array_equal(ok[sel], ook), (N, K, L)
    plan.close()
    for c in codes:
        c.close()
