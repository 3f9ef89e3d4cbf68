"""GPU parity: the CUDA decoder (through the C ABI) against the CPU oracle.

Payload bits, winning slot and CRC flag must be identical; the penalty must
be identical for int8 LLRs (exact integers) and within 1e-5 relative for
float32 (the float sums follow the same canonical order on both sides, so
they are expected to be identical too).
"""
import os

import numpy as np
import pytest

from paper_1505_01466_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1
MODES = {"SPC_MAX_4": 0, "SPC_ANY": 1, "NO_SPECIAL_NODES": 2}
OMODE = {0: 0, 1: 1, 2: 2}   # library mode -> oracle mode (same numbering)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def gpu_decode(torch, code, llr_np):
    llr = torch.from_numpy(np.ascontiguousarray(llr_np)).cuda()
    bits, pm, ok, slot = code.decode(llr)
    torch.cuda.synchronize()
    return bits.cpu().numpy(), pm.cpu().numpy(), ok.cpu().numpy(), slot.cpu().numpy()


def assert_parity(g, o, dtype, what=""):
    gb, gpm, gok, gsl = g
    ob, opm, ook, osl = o
    bad = np.flatnonzero((gb != ob).any(axis=1) | (gsl != osl) | (gok != ook))
    assert bad.size == 0, f"{what}: {bad.size} frames differ, first {bad[:8]}"
    if dtype == "i8":
        assert np.array_equal(gpm, opm), what
    else:
        np.testing.assert_allclose(gpm, opm, rtol=1e-5, atol=0, err_msg=what)


def run_case(torch, oracle_mod, frozen, crc_len, poly, L, llr_np, mode=0, launch=None):
    from paper_1505_01466_gb300.polar import PolarCode
    code = PolarCode(frozen, crc_len, poly, L, mode=mode)
    if launch is not None:
        code.set_launch(1 if llr_np.dtype == np.int8 else 0, *launch)
    g = gpu_decode(torch, code, llr_np)
    o = oracle_mod.decode(frozen, L, llr_np, crc_len, poly, OMODE[mode], n_threads=NT)
    code.close()
    return g, o


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_config_256_128_crc8_L4_all_frames(torch_cuda, oracle_mod, dtype):
    # (256,128) CRC-8 L=4, GA design 2 dB, Eb/N0 2.5 dB, 10^4 frames.
    fr = I.ga_frozen_mask(256, 128, 2.0, 120 / 256)
    f = I.make_frames(fr, 8, I.CRC8_POLY, 2.5, 10000, seed=101)
    llr = f.llr_i8 if dtype == "i8" else f.llr_f32
    g, o = run_case(torch_cuda, oracle_mod, fr, 8, I.CRC8_POLY, 4, llr)
    assert_parity(g, o, dtype, "(256,128) L=4")


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("mode", list(MODES))
def test_random_codes_all_list_sizes(torch_cuda, oracle_mod, dtype, mode):
    rng = np.random.default_rng(hash((dtype, mode)) % 2 ** 32)
    for N in (8, 16, 32, 64, 128, 512):
        for L in (1, 2, 4, 8, 16, 32):
            K = int(rng.integers(max(2, N // 8), N))
            crc = 8 if K > 12 else 0
            fr = I.ga_frozen_mask(N, K, float(rng.uniform(0, 4)), max(K - crc, 1) / N)
            snr = float(rng.uniform(-1.0, 3.0))
            f = I.make_frames(fr, crc, I.CRC8_POLY, snr, 24, seed=int(rng.integers(1 << 30)))
            llr = f.llr_i8 if dtype == "i8" else f.llr_f32
            g, o = run_case(torch_cuda, oracle_mod, fr, crc, I.CRC8_POLY, L, llr, MODES[mode])
            assert_parity(g, o, dtype, f"N={N} K={K} L={L} mode={mode}")


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("L", [2, 4, 8, 32])
def test_config_1024_860_crc32_sampled(torch_cuda, oracle_mod, dtype, L):
    fr = I.ga_frozen_mask(1024, 860, 4.0, 828 / 1024)
    for snr in (3.5, 4.5):
        f = I.make_frames(fr, 32, I.CRC32_POLY, snr, 256 if L < 32 else 96, seed=int(snr * 100) + L)
        llr = f.llr_i8 if dtype == "i8" else f.llr_f32
        g, o = run_case(torch_cuda, oracle_mod, fr, 32, I.CRC32_POLY, L, llr)
        assert_parity(g, o, dtype, f"(1024,860) L={L} {snr} dB")


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("L", [8, 32])
def test_config_2048_1723_crc32_sampled(torch_cuda, oracle_mod, dtype, L):
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.5, 64, seed=2048 + L)
    llr = f.llr_i8 if dtype == "i8" else f.llr_f32
    g, o = run_case(torch_cuda, oracle_mod, fr, 32, I.CRC32_POLY, L, llr)
    assert_parity(g, o, dtype, f"(2048,1723) L={L}")


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_launch_shapes_and_spills_agree(torch_cuda, oracle_mod, dtype):
    fr = I.ga_frozen_mask(1024, 512, 2.0, 480 / 1024)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 1.5, 48, seed=77)
    llr = f.llr_i8 if dtype == "i8" else f.llr_f32
    o = oracle_mod.decode(fr, 16, llr, 32, I.CRC32_POLY, 0, n_threads=NT)
    from paper_1505_01466_gb300.polar import PolarCode
    for warps in (1, 2, 4):
        for budget in (0, 60000, 20000):
            for cta in (128, 512):
                code = PolarCode(fr, 32, I.CRC32_POLY, 16)
                try:
                    code.set_launch(1 if dtype == "i8" else 0, warps, budget, cta)
                except Exception:
                    continue
                g = gpu_decode(torch_cuda, code, llr)
                assert_parity(g, o, dtype, f"warps={warps} budget={budget} cta={cta} info={code.info()}")


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_edge_cases(torch_cuda, oracle_mod, dtype):
    from paper_1505_01466_gb300.polar import PolarCode
    rng = np.random.default_rng(5)
    cases = []
    # rate-1 code (root is a Rate-1 leaf), repetition code (root is a Rep leaf)
    cases.append((np.zeros(32, np.uint8), 0))
    cases.append((np.array([1] * 63 + [0], np.uint8), 0))
    # single-parity-check code of length 4 under SPC_ANY handled by mode below
    cases.append((I.ga_frozen_mask(128, 64, 1.0), 8))
    for fr, crc in cases:
        N = fr.size
        llrs = [np.zeros((4, N), np.float32),                         # all-zero LLRs: ties everywhere
                -np.ones((4, N), np.float32) * 3,                    # all negative
                rng.integers(-2, 3, (16, N)).astype(np.float32),     # many ties
                rng.normal(0, 40, (16, N)).astype(np.float32)]      # saturating in int8
        for x in llrs:
            llr = I.quantize_i8(x / 4.0) if dtype == "i8" else x
            for L in (1, 2, 8, 32):
                for mode in (0, 1, 2):
                    g, o = run_case(torch_cuda, oracle_mod, fr, crc, I.CRC8_POLY, L, llr, mode)
                    assert_parity(g, o, dtype, f"edge N={N} L={L} mode={mode}")
    # -128 in int8 input is read as -127
    if dtype == "i8":
        fr = I.ga_frozen_mask(64, 32, 1.0)
        x = rng.integers(-128, 128, (8, 64)).astype(np.int8)
        g, o = run_case(torch_cuda, oracle_mod, fr, 0, 0, 4, x)
        assert_parity(g, o, dtype, "-128 input")
    # zero frames is a no-op
    code = PolarCode(I.ga_frozen_mask(64, 32, 1.0), 0, 0, 4)
    t = torch_cuda.zeros((0, 64), dtype=torch_cuda.float32, device="cuda")
    code.decode(t)


def test_deterministic_and_stream_safe(torch_cuda, oracle_mod):
    from paper_1505_01466_gb300.polar import PolarCode
    fr = I.ga_frozen_mask(1024, 860, 4.0, 828 / 1024)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.5, 2000, seed=9)
    code = PolarCode(fr, 32, I.CRC32_POLY, 8)
    llr = torch_cuda.from_numpy(f.llr_f32).cuda()
    ref = code.decode(llr)
    s1, s2 = torch_cuda.cuda.Stream(), torch_cuda.cuda.Stream()
    outs = []
    for s in (s1, s2, s1, s2):
        with torch_cuda.cuda.stream(s):
            outs.append(code.decode(llr, stream=s))
    torch_cuda.cuda.synchronize()
    for out in outs:
        for a, b in zip(out, ref):
            assert torch_cuda.equal(a, b)


def test_autotune_keeps_results(torch_cuda, oracle_mod):
    from paper_1505_01466_gb300.polar import PolarCode
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.75, 1024, seed=31)
    for llr_np in (f.llr_f32, f.llr_i8):
        code = PolarCode(fr, 32, I.CRC32_POLY, 8)
        llr = torch_cuda.from_numpy(llr_np).cuda()
        before = code.decode(llr)
        w, b, t = code.autotune(llr)
        assert w in (1, 2, 4) and t in (128, 256, 512)
        after = code.decode(llr)
        torch_cuda.cuda.synchronize()
        for x, y in zip(before, after):
            assert torch_cuda.equal(x, y)
        o = oracle_mod.decode(fr, 8, llr_np[:64], 32, I.CRC32_POLY, 0, n_threads=NT)
        assert_parity(tuple(t[:64].cpu().numpy() for t in after), o, "i8" if llr_np.dtype == np.int8 else "f32")


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("n_frames", [10001, 70001])
def test_host_buffer_decode_matches_device_decode(torch_cuda, oracle_mod, dtype, n_frames):
    # polar_list_decode_host: chunked copy in / decode / copy out, chunks growing
    # from the first (2048 frames) to the largest, ragged last chunk
    from paper_1505_01466_gb300.polar import PolarCode
    torch = torch_cuda
    fr = I.ga_frozen_mask(512, 300, 3.0, 268 / 512)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 2.5, n_frames, seed=12)
    x = f.llr_i8 if dtype == "i8" else f.llr_f32
    code = PolarCode(fr, 32, I.CRC32_POLY, 8)
    ref = [t.cpu() for t in code.decode(torch.from_numpy(x).cuda())]
    for pinned in (True, False):
        hl = torch.from_numpy(x).clone()
        if pinned:
            hl = hl.pin_memory()
        bits = torch.full_like(ref[0], 0xAA)
        pm = torch.full_like(ref[1], -1.0)
        ok = torch.full_like(ref[2], 7)
        slot = torch.full_like(ref[3], -1)
        code.decode_host(hl, bits, pm, ok, slot)
        for a, b in zip((bits, pm, ok, slot), ref):
            assert torch.equal(a, b)
    o = oracle_mod.decode(fr, 8, x[-40:], 32, I.CRC32_POLY, 0, n_threads=NT)
    assert_parity(tuple(t[-40:].numpy() for t in ref), o, dtype, "host decode tail")
    code.close()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("case", [(256, 128, 8, 4, 2.0, 2.0), (1024, 860, 32, 8, 4.0, 3.25), (2048, 1723, 32, 32, 4.0, 3.5)])
def test_systematic_codes(torch_cuda, oracle_mod, dtype, case):
    from paper_1505_01466_gb300.polar import PolarCode
    N, K, crc, L, design, snr = case
    poly = I.CRC8_POLY if crc == 8 else I.CRC32_POLY
    fr = I.ga_frozen_mask(N, K, design, (K - crc) / N)
    f = I.make_frames(fr, crc, poly, snr, 200 if N < 2048 else 64, seed=N + L, systematic=True)
    llr = f.llr_i8 if dtype == "i8" else f.llr_f32
    for mode in (0, 2):
        code = PolarCode(fr, crc, poly, L, mode=mode, systematic=True)
        g = gpu_decode(torch_cuda, code, llr)
        code.close()
        o = oracle_mod.decode(fr, L, llr, crc, poly, mode | oracle_mod.SYSTEMATIC, n_threads=NT)
        assert_parity(g, o, dtype, f"systematic ({N},{K}) L={L} mode={mode}")
        # most frames decode to their payload
        got = I.unpack_bits_lsb(g[0], K - crc)
        assert (got == f.payload).all(axis=1).mean() > 0.5


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_full_size_in_the_benchmark_launch_configuration(torch_cuda, oracle_mod, dtype):
    # (2048,1723) L=32 at 4 dB, 2^20 frames in HBM, the autotuned launch shape the
    # benchmark times: 4096 distinct frames tiled 256 times. Every copy of a frame
    # must decode like the first one (the whole batch is checked), and a sample of
    # the distinct frames, including the last ones, against the oracle.
    from paper_1505_01466_gb300.polar import PolarCode
    torch = torch_cuda
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    f = I.make_frames_chunked(fr, 32, I.CRC32_POLY, 4.0, 4096, seed=2020)
    x = torch.from_numpy(f.llr_i8 if dtype == "i8" else f.llr_f32).cuda()
    llr = x.repeat(256, 1)
    code = PolarCode(fr, 32, I.CRC32_POLY, 32)
    code.autotune(llr[:16384])
    bits, pm, ok, slot = code.decode(llr)
    torch.cuda.synchronize()
    for t in (bits, pm, ok, slot):
        v = t.view(256, 4096, -1)
        assert torch.equal(v, v[:1].expand_as(v))
    sample = np.r_[0:24, 4096 - 24:4096]
    src = (f.llr_i8 if dtype == "i8" else f.llr_f32)[sample]
    o = oracle_mod.decode(fr, 32, src, 32, I.CRC32_POLY, 0, n_threads=NT)
    last = slice(llr.shape[0] - 4096, llr.shape[0])
    g = tuple(t[last][torch.from_numpy(sample).cuda()].cpu().numpy() for t in (bits, pm, ok, slot))
    assert_parity(g, o, dtype, "full size, sampled")
    code.close()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_small_batches_take_the_latency_shape(torch_cuda, oracle_mod, dtype):
    # at most one frame per SM: four warps and a CTA's shared memory per frame;
    # a fixed shape (set_launch) is kept, and the results never depend on it
    from paper_1505_01466_gb300.polar import PolarCode
    torch = torch_cuda
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.5, 100, seed=55)
    x = torch.from_numpy(f.llr_i8 if dtype == "i8" else f.llr_f32).cuda()
    code = PolarCode(fr, 32, I.CRC32_POLY, 32)
    small = [t.cpu() for t in code.decode(x)]                      # latency shape
    code.set_launch(1 if dtype == "i8" else 0, 1, 7000, 512)        # fixed shape from now on
    fixed = [t.cpu() for t in code.decode(x)]
    for a, b in zip(small, fixed):
        assert torch.equal(a, b)
    o = oracle_mod.decode(fr, 32, (f.llr_i8 if dtype == "i8" else f.llr_f32)[:24], 32, I.CRC32_POLY, 0,
                          n_threads=NT)
    assert_parity(tuple(t[:24].numpy() for t in small), o, dtype, "latency shape")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    code.autotune(x.repeat(64, 1))                                  # autotune lifts the fix
    ev0.record()
    code.decode(x[:1])
    ev1.record()
    torch.cuda.synchronize()
    assert ev0.elapsed_time(ev1) < 50.0
    code.close()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("L", [32, 128])
def test_maximum_sizes(torch_cuda, oracle_mod, dtype, L):
    # the largest code length (4096) with the largest narrow and wide lists
    fr = I.ga_frozen_mask(4096, 3686, 4.0, 3654 / 4096)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.5, 24 if L == 32 else 8, seed=4096 + L)
    llr = f.llr_i8 if dtype == "i8" else f.llr_f32
    g, o = run_case(torch_cuda, oracle_mod, fr, 32, I.CRC32_POLY, L, llr)
    assert_parity(g, o, dtype, f"(4096,3686) L={L}")
