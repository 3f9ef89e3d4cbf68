"""GPU parity of the L = 1 (Fast-SSC) kernels against the oracle.

A code with L = 1 runs its own kernels unless set_launch fixes a shape of the
list kernels: one lane per frame (32 frames per warp) for batches larger than
the SM count, one warp per frame for smaller ones. All three must give the
oracle's results bit for bit (payload, CRC flag, slot 0) with the penalty
exact for int8 and within 1e-5 relative for float32.
"""
import os

import numpy as np
import pytest

from paper_1505_01466_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _decode(torch, code, llr, offset=0):
    """Decode through polar_list_decode; offset > 0 starts the LLR rows that
    many elements past an aligned allocation."""
    flat = torch.empty(llr.size + offset, dtype=torch.from_numpy(llr[:0]).dtype, device="cuda")
    view = flat[offset:].view(llr.shape)
    view.copy_(torch.from_numpy(np.ascontiguousarray(llr)))
    bits, pm, ok, slot = code.decode(view)
    torch.cuda.synchronize()
    return bits.cpu().numpy(), pm.cpu().numpy(), ok.cpu().numpy(), slot.cpu().numpy()


def _check(g, o, dtype, what):
    gb, gpm, gok, gsl = g
    ob, opm, ook, osl = o
    bad = np.flatnonzero((gb != ob).any(axis=1) | (gsl != osl) | (gok != ook))
    assert bad.size == 0, f"{what}: {bad.size} frames differ, first {bad[:8]}"
    assert (gsl == 0).all()
    if dtype == "i8":
        assert np.array_equal(gpm, opm), what
    else:
        np.testing.assert_allclose(gpm, opm, rtol=1e-5, atol=0, err_msg=what)


def _both_kernels(torch, oracle_mod, fr, crc, poly, llr, mode=0, systematic=False, offset=0):
    """The three decoders of an L = 1 code: a batch larger than the SM count
    takes the lane-per-frame kernel, a batch no larger the warp-per-frame
    kernel, and an explicit launch shape the list kernel at L = 1."""
    from paper_1505_01466_gb300.polar import PolarCode
    dtype = "i8" if llr.dtype == np.int8 else "f32"
    o = oracle_mod.decode(fr, 1, llr, crc, poly, mode | (oracle_mod.SYSTEMATIC if systematic else 0), n_threads=NT)
    code = PolarCode(fr, crc, poly, 1, mode=mode, systematic=systematic)
    info = code.info()
    assert info["warps_per_frame"] == [1, 1] and info["frames_per_cta"][0] % 32 == 0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    reps = -(-(sms + 1) // llr.shape[0])
    g = _decode(torch, code, np.concatenate([llr] * reps), offset)
    _check(g, tuple(np.concatenate([x] * reps) for x in o), dtype,
           f"lane per frame N={fr.size} mode={mode} sys={systematic} offset={offset}")
    m = min(llr.shape[0], sms, 100)
    g = _decode(torch, code, llr[:m], offset)
    _check(g, tuple(x[:m] for x in o), dtype, f"warp per frame N={fr.size} mode={mode} sys={systematic} offset={offset}")
    code.set_launch(1 if dtype == "i8" else 0, 1, 0, 128)          # the list kernel at L = 1
    g2 = _decode(torch, code, llr, offset)
    _check(g2, o, dtype, f"list kernel N={fr.size} mode={mode}")
    code.close()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_random_codes_every_length(torch_cuda, oracle_mod, dtype, mode):
    rng = np.random.default_rng(1000 + 10 * mode + (dtype == "i8"))
    for N in (8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096):   # the library takes N >= 8
        K = int(rng.integers(1, N + 1))
        crc = 8 if K > 12 else 0
        fr = I.ga_frozen_mask(N, K, float(rng.uniform(0, 4)), max(K - crc, 1) / N)
        f = I.make_frames(fr, crc, I.CRC8_POLY, float(rng.uniform(-1, 4)), 40 if N >= 1024 else 96,
                          seed=int(rng.integers(1 << 30)))
        llr = f.llr_i8 if dtype == "i8" else f.llr_f32
        _both_kernels(torch_cuda, oracle_mod, fr, crc, I.CRC8_POLY, llr, mode)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_bench_code_crc32_and_systematic(torch_cuda, oracle_mod, dtype):
    for N, K, design, snr in ((2048, 1723, 4.0, 3.5), (1024, 860, 4.0, 3.0)):
        fr = I.ga_frozen_mask(N, K, design, (K - 32) / N)
        for systematic in (False, True):
            f = I.make_frames(fr, 32, I.CRC32_POLY, snr, 300, seed=N + systematic, systematic=systematic)
            llr = f.llr_i8 if dtype == "i8" else f.llr_f32
            _both_kernels(torch_cuda, oracle_mod, fr, 32, I.CRC32_POLY, llr, 0, systematic)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_unaligned_rows_and_adversarial_values(torch_cuda, oracle_mod, dtype):
    """Rows that start off a 16-byte boundary take the scalar loads; ties,
    zeros (and -0.0), saturation and -128 exercise every comparison."""
    fr = I.ga_frozen_mask(1024, 700, 2.0, 692 / 1024)
    rng = np.random.default_rng(9)
    n = 64
    if dtype == "i8":
        llr = rng.choice(np.array([-128, -127, -1, 0, 1, 2, 127], np.int8), size=(n, 1024))
        llr[:8] = rng.integers(-128, 128, (8, 1024), dtype=np.int16).astype(np.int8)
        llr[8:12] = 0
        llr[12:16] = -128
    else:
        llr = rng.choice(np.array([-2.0, -0.5, -0.0, 0.0, 0.5, 2.0], np.float32), size=(n, 1024))
        llr[8:12] = 0.0
        llr[12:16] = -0.0
        llr[16:24] = rng.normal(0, 3, (8, 1024)).astype(np.float32)
    for offset in (0, 1, 3):
        _both_kernels(torch_cuda, oracle_mod, fr, 8, I.CRC8_POLY, llr, 0, False, offset)


def test_empty_and_single_frames(torch_cuda, oracle_mod):
    from paper_1505_01466_gb300.polar import PolarCode
    fr = I.ga_frozen_mask(512, 300, 2.0, 292 / 512)
    code = PolarCode(fr, 8, I.CRC8_POLY, 1)
    torch = torch_cuda
    bits, pm, ok, slot = code.decode(torch.empty((0, 512), dtype=torch.float32, device="cuda"))
    assert bits.shape[0] == 0
    f = I.make_frames(fr, 8, I.CRC8_POLY, 2.0, 3, seed=4)
    o = oracle_mod.decode(fr, 1, f.llr_f32, 8, I.CRC8_POLY, 0, n_threads=NT)
    for i in range(3):
        g = _decode(torch, code, f.llr_f32[i:i + 1])
        _check(g, tuple(x[i:i + 1] for x in o), "f32", f"frame {i}")
    code.close()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_codes_whose_root_is_a_leaf(torch_cuda, oracle_mod, dtype):
    """Rate-1, repetition and (under SPC_ANY) SPC codes: the leaf reads the
    channel row itself, which the kernel copies to shared memory first."""
    rng = np.random.default_rng(31)
    for N in (8, 64, 4096):
        rate1 = np.zeros(N, np.uint8)
        rep = np.ones(N, np.uint8)
        rep[-1] = 0
        spc = np.zeros(N, np.uint8)
        spc[0] = 1
        for fr, mode in ((rate1, 0), (rep, 0), (spc, 1), (rate1, 2)):
            llr = rng.normal(0.5, 2.0, (48, N)).astype(np.float32)
            if dtype == "i8":
                llr = I.quantize_i8(llr)
                llr[:4, :3] = -128
            _both_kernels(torch_cuda, oracle_mod, fr, 0, 0, llr, mode)


def test_sync_waits_for_the_stream(torch_cuda, oracle_mod):
    """polar_sync waits for a decode enqueued on a side stream and reports no
    error; the outputs are complete afterwards without any other wait."""
    from paper_1505_01466_gb300 import polar
    torch = torch_cuda
    fr = I.ga_frozen_mask(1024, 860, 4.0, 828 / 1024)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.5, 512, seed=12)
    o = oracle_mod.decode(fr, 1, f.llr_f32, 32, I.CRC32_POLY, 0, n_threads=NT)
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 1)
    side = torch.cuda.Stream()
    llr = torch.from_numpy(f.llr_f32).cuda()
    torch.cuda.synchronize()
    bits = torch.empty((512, 104), dtype=torch.uint8, device="cuda")
    pm = torch.empty(512, dtype=torch.float32, device="cuda")
    ok = torch.empty(512, dtype=torch.uint8, device="cuda")
    slot = torch.empty(512, dtype=torch.int32, device="cuda")
    code.decode_into(llr, bits, pm, ok, slot, stream=side)
    polar.sync(side)
    g = tuple(t.cpu().numpy() for t in (bits, pm, ok, slot))
    _check(g, o, "f32", "after polar_sync")
    polar.sync()                                        # the current stream: nothing pending
    code.close()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_every_shared_memory_budget(torch_cuda, oracle_mod, dtype):
    """The L = 1 kernel keeps the lowest alpha stages of its 32 frames per warp
    in shared memory up to a budget and the others in global scratch: from
    every stage on chip (int8) down to none (budget 1), the results are the
    oracle's. The scratch is poisoned, so a value read before it is written
    would show up."""
    from paper_1505_01466_gb300 import polar
    torch = torch_cuda
    lib = polar.load_library()
    dt = polar.LLR_I8 if dtype == "i8" else polar.LLR_F32
    rng = np.random.default_rng(5)
    for N, K, crc in ((2048, 1723, 32), (4096, 2500, 8), (64, 40, 8)):
        poly = I.CRC32_POLY if crc == 32 else I.CRC8_POLY
        fr = I.ga_frozen_mask(N, K, 3.0, (K - crc) / N)
        f = I.make_frames(fr, crc, poly, float(rng.uniform(2.0, 3.5)), 200, seed=N)
        llr = f.llr_i8 if dtype == "i8" else f.llr_f32
        o = oracle_mod.decode(fr, 1, llr, crc, poly, 0, n_threads=NT)
        code = polar.PolarCode(fr, crc, poly, 1)
        splits = set()
        lib.polar_debug_inject(polar.INJECT_POISON, 1)
        try:
            for budget in (0, 232448, 100000, 60000, 30000, 12000, 1):
                code.set_smem_budget(dt, budget)
                info = code.info()
                splits.add(info["spill_mask"][dt])
                g = _decode(torch, code, llr)
                _check(g, o, dtype, f"N={N} budget={budget}")
        finally:
            lib.polar_debug_inject(polar.INJECT_POISON, 0)
        assert ((1 << fr.size.bit_length() - 1) - 1) in splits          # every stage in scratch once
        assert len(splits) >= (3 if N >= 1024 else 2)
        code.close()


def test_autotune_keeps_results(torch_cuda, oracle_mod):
    from paper_1505_01466_gb300 import polar
    torch = torch_cuda
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.5, 1000, seed=3)
    o = oracle_mod.decode(fr, 1, f.llr_f32, 32, I.CRC32_POLY, 0, n_threads=NT)
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 1)
    w, b, t = code.autotune(torch.from_numpy(f.llr_f32).cuda())
    assert w == 1 and t % 32 == 0 and b == 0          # a 1000-frame sample keeps the default
    _check(_decode(torch, code, f.llr_f32), o, "f32", "after autotune")
    code.close()
