"""The allocation-free decode entry point (polar_list_decode_noalloc).

It is meant for callers that cannot allocate device memory while they
decode -- real-time paths that may not take allocator locks or run out of
memory once running, and hosts with a fixed memory budget. It must return
exactly what the ordinary entry point returns. This file is collected last
so that a run stopping at the first failure has already run every other
test.
"""
import ctypes

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


def _call(torch, polar, fn, code, llr, dt):
    F = llr.shape[0]
    kb = (code.k + 7) // 8
    bits = torch.full((F, kb), 0xAA, dtype=torch.uint8, device="cuda")
    pm = torch.full((F,), -1.0, dtype=torch.float32, device="cuda")
    ok = torch.full((F,), 7, dtype=torch.uint8, device="cuda")
    slot = torch.full((F,), -1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = fn(code.handle, ctypes.c_void_p(llr.data_ptr()), dt, F, ctypes.c_void_p(bits.data_ptr()),
            ctypes.c_void_p(pm.data_ptr()), ctypes.c_void_p(ok.data_ptr()), ctypes.c_void_p(slot.data_ptr()), stream)
    assert st == 0, polar.load_library().polar_strerror(st)
    torch.cuda.synchronize()
    return bits.cpu(), pm.cpu(), ok.cpu(), slot.cpu()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_noalloc_matches_ordinary_decode_twice(env, dtype):
    torch, polar = env
    lib = polar.load_library()
    assert lib.polar_noalloc_scratch_bytes() == 64 << 20
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.75, 3000, seed=404)
    x = f.llr_i8 if dtype == "i8" else f.llr_f32
    dt = polar.LLR_I8 if dtype == "i8" else polar.LLR_F32
    llr = torch.from_numpy(x).cuda()
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 32)
    # a shape that keeps alpha stages in global scratch, so the fixed array is used
    code.set_launch(dt, 4, 40000)
    assert code.info()["scratch_per_frame"][dt] > 0
    ref = _call(torch, polar, lib.polar_list_decode, code, llr, dt)
    for _ in range(2):      # two calls in a row share the array
        got = _call(torch, polar, lib.polar_list_decode_noalloc, code, llr, dt)
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    code.close()


def test_noalloc_small_code_without_scratch(env):
    torch, polar = env
    lib = polar.load_library()
    fr = I.ga_frozen_mask(256, 128, 2.0, 120 / 256)
    f = I.make_frames(fr, 8, I.CRC8_POLY, 2.5, 500, seed=5)
    llr = torch.from_numpy(f.llr_f32).cuda()
    code = polar.PolarCode(fr, 8, I.CRC8_POLY, 4)
    ref = _call(torch, polar, lib.polar_list_decode, code, llr, polar.LLR_F32)
    for _ in range(2):
        got = _call(torch, polar, lib.polar_list_decode_noalloc, code, llr, polar.LLR_F32)
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    code.close()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_noalloc_l1_code(env, dtype):
    """An L = 1 code runs its own kernel, which needs no scratch, through the
    allocation-free entry point too; with a list-kernel shape fixed it goes
    through the fixed array like any list code. All four agree."""
    torch, polar = env
    lib = polar.load_library()
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.5, 2000, seed=41)
    x = f.llr_i8 if dtype == "i8" else f.llr_f32
    dt = polar.LLR_I8 if dtype == "i8" else polar.LLR_F32
    llr = torch.from_numpy(x).cuda()
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 1)
    ref = _call(torch, polar, lib.polar_list_decode, code, llr, dt)
    got = _call(torch, polar, lib.polar_list_decode_noalloc, code, llr, dt)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    code.set_launch(dt, 1, 2000, 512)                      # small enough to spill for both dtypes
    assert code.info()["scratch_per_frame"][dt] > 0
    for fn in (lib.polar_list_decode, lib.polar_list_decode_noalloc):
        got = _call(torch, polar, fn, code, llr, dt)
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    code.close()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_noalloc_cuts_the_grid_to_the_array(env, dtype):
    """Every alpha stage spilled (a 3000-byte shared-memory budget): a full
    grid of this shape needs more scratch than the fixed array holds, so the
    call launches fewer persistent CTAs; every frame still decodes alike."""
    torch, polar = env
    lib = polar.load_library()
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    f = I.make_frames(fr, 32, I.CRC32_POLY, 3.75, 1500, seed=77)
    x = f.llr_i8 if dtype == "i8" else f.llr_f32
    dt = polar.LLR_I8 if dtype == "i8" else polar.LLR_F32
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 32)
    code.set_launch(dt, 1, 3000, 512)          # room for the path tables only
    code.set_recompute(dt, 0)                  # every alpha stage stored
    info = code.info()
    per_cta = info["scratch_per_frame"][dt] * info["frames_per_cta"][dt]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fit = lib.polar_noalloc_scratch_bytes() // per_cta
    assert per_cta * sms > lib.polar_noalloc_scratch_bytes()        # the full grid would not fit
    reps = (fit + 4) * info["frames_per_cta"][dt] // x.shape[0] + 1   # more frames than the cut grid holds at once
    llr = torch.from_numpy(np.tile(x, (reps, 1))).cuda()
    assert llr.shape[0] > fit * info["frames_per_cta"][dt]
    ref = _call(torch, polar, lib.polar_list_decode, code, llr, dt)
    for _ in range(2):
        got = _call(torch, polar, lib.polar_list_decode_noalloc, code, llr, dt)
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    code.close()


def test_noalloc_refuses_wide_codes(env):
    torch, polar = env
    lib = polar.load_library()
    fr = I.ga_frozen_mask(256, 128, 2.0, 120 / 256)
    code = polar.PolarCode(fr, 8, I.CRC8_POLY, 64)
    llr = torch.zeros((4, 256), dtype=torch.float32, device="cuda")
    kb = (code.k + 7) // 8
    bits = torch.zeros((4, kb), dtype=torch.uint8, device="cuda")
    pm = torch.zeros(4, dtype=torch.float32, device="cuda")
    st = lib.polar_list_decode_noalloc(code.handle, ctypes.c_void_p(llr.data_ptr()), polar.LLR_F32, 4,
                                       ctypes.c_void_p(bits.data_ptr()), ctypes.c_void_p(pm.data_ptr()),
                                       None, None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -4                                                 # POLAR_EUNSUPPORTED
    code.close()
