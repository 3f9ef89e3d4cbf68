"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, validates its arguments, and builds the same decoding
schedule as the oracle (host code only, POLAR_HOST_ONLY codes)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1505_01466_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def polar():
    from paper_1505_01466_gb300 import build
    build.build()
    import paper_1505_01466_gb300.polar as polar
    polar.load_library()
    return polar


def _declared_symbols():
    syms = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            syms |= set(re.findall(r"POLAR_API\s+[\w\s\*]*?\b(polar_\w+)\s*\(", text))
    return syms


def test_library_exports_every_declared_symbol(polar):
    lib = polar.load_library()
    declared = _declared_symbols()
    assert "polar_list_decode" in declared and "polar_code_create" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(polar.EXPORTED)


def test_strerror(polar):
    lib = polar.load_library()
    for st in range(0, -7, -1):
        assert lib.polar_strerror(st)
    assert lib.polar_strerror(-99) == b"unknown status"


def _create(polar, N, K, mask, crc_len=0, poly=0, L=4, flags=0):
    h = ctypes.c_void_p()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    st = polar.load_library().polar_code_create(ctypes.byref(h), N, K, m.ctypes.data_as(ctypes.c_void_p),
                                               crc_len, poly, L, flags | polar.HOST_ONLY)
    if st == 0:
        polar.load_library().polar_code_destroy(h)
    else:
        assert not h.value
    return st


def test_create_validation(polar):
    fr = I.ga_frozen_mask(64, 32, 2.0)
    assert _create(polar, 64, 32, fr) == polar.POLAR_OK
    assert _create(polar, 63, 32, fr[:63]) == polar.POLAR_EINVAL      # not a power of two
    assert _create(polar, 4, 2, fr[:4]) == polar.POLAR_EINVAL          # N < 8
    assert _create(polar, 64, 31, fr) == polar.POLAR_EINVAL            # mask has N-K ones
    assert _create(polar, 64, 32, fr, crc_len=32) == polar.POLAR_EINVAL  # crc_len >= K
    assert _create(polar, 64, 32, fr, crc_len=33) == polar.POLAR_EINVAL
    assert _create(polar, 64, 32, fr, L=3) == polar.POLAR_EUNSUPPORTED
    assert _create(polar, 64, 32, fr, L=64) == polar.POLAR_OK             # the wide kernel
    assert _create(polar, 64, 32, fr, L=256) == polar.POLAR_EUNSUPPORTED
    assert _create(polar, 64, 32, fr, flags=7) == polar.POLAR_EINVAL
    h = ctypes.c_void_p()
    assert polar.load_library().polar_code_create(None, 64, 32, fr.ctypes.data_as(ctypes.c_void_p), 0, 0, 4, 0) \
        == polar.POLAR_EINVAL
    assert polar.load_library().polar_code_create(ctypes.byref(h), 64, 32, None, 0, 0, 4, 0) == polar.POLAR_EINVAL
    assert polar.load_library().polar_code_destroy(None) == polar.POLAR_OK


def test_decode_rejects_host_only_and_bad_args(polar):
    fr = I.ga_frozen_mask(64, 32, 2.0)
    code = polar.PolarCode(fr, 8, I.CRC8_POLY, 4, host_only=True)
    lib = polar.load_library()
    st = lib.polar_list_decode(code.handle, ctypes.c_void_p(16), 0, 1, ctypes.c_void_p(16), ctypes.c_void_p(16),
                               None, None, None)
    assert st == polar.POLAR_EINVAL
    assert lib.polar_list_decode(None, None, 0, 1, None, None, None, None, None) == polar.POLAR_EINVAL


@pytest.mark.parametrize("mode", ["SPC_MAX_4", "SPC_ANY", "NO_SPECIAL_NODES"])
def test_schedule_matches_oracle(polar, oracle_mod, mode):
    omode = {"SPC_MAX_4": oracle_mod.SPC4, "SPC_ANY": oracle_mod.SPC_ANY,
             "NO_SPECIAL_NODES": oracle_mod.BITWISE}[mode]
    rng = np.random.default_rng(8)
    for _ in range(30):
        N = int(rng.choice([8, 16, 64, 256, 1024]))
        K = int(rng.integers(1, N + 1))
        fr = np.ones(N, np.uint8)
        fr[rng.choice(N, K, replace=False)] = 0
        code = polar.PolarCode(fr, 0, 0, 4, mode=getattr(polar, mode), host_only=True)
        assert code.schedule() == oracle_mod.schedule(fr, omode)
    for N, K, d, r in [(256, 128, 2.0, 120 / 256), (1024, 860, 4.0, 828 / 1024), (2048, 1723, 4.0, 1691 / 2048)]:
        fr = I.ga_frozen_mask(N, K, d, r)
        code = polar.PolarCode(fr, 32, I.CRC32_POLY, 32, mode=getattr(polar, mode), host_only=True)
        assert code.schedule() == oracle_mod.schedule(fr, omode)


def test_code_info_and_op_count(polar):
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 32, host_only=True)
    info = code.info()
    assert info["n_leaves"] == info["n_rate0"] + info["n_rate1"] + info["n_rep"] + info["n_spc"]
    assert info["k"] == 1691
    # every leaf is one entry, every inner node three (F, G, Combine)
    assert info["n_ops"] == info["n_leaves"] + 3 * (info["n_leaves"] - 1)
    # shared memory per frame fits a CTA; larger stages spilled to global scratch
    for d in (0, 1):
        assert info["smem_per_frame"][d] * info["frames_per_cta"][d] <= 232448
    assert code.op_count() > 2048 * 11  # at least one path's F/G work
    # a smaller budget moves more alpha stages to global scratch
    code.set_launch(1, 4, 20000)
    assert code.info()["smem_per_frame"][1] <= 20000
    assert code.info()["spill_mask"][1] != 0
    with pytest.raises(polar.PolarError):
        code.set_launch(1, 3, 0)


def test_fer_statistics_helpers():
    import bench
    lo, hi = bench.clopper_pearson(0, 100)
    assert lo == 0.0 and hi == pytest.approx(1 - 0.005 ** (1 / 100))   # closed form at x = 0
    lo, hi = bench.clopper_pearson(50, 100)
    assert lo < 0.5 < hi and lo == pytest.approx(1 - hi)               # symmetric at x = n/2
    a = np.zeros(1000, bool); a[:120] = True
    b = a.copy(); b[0] = False; b[500] = True
    t = bench.paired_fer_test(a, b)
    assert t["errors"] == [120, 120] and t["only_first_failed"] == 1 and t["match"] and not t["underpowered"]
    c = np.zeros(1000, bool); c[:10] = True
    assert not bench.paired_fer_test(a, c)["match"]


def test_binding_fails_loudly_without_the_library(tmp_path):
    # the product path has no CPU fallback: a missing library is an ImportError
    import subprocess
    import sys
    code = ("import paper_1505_01466_gb300.polar as p\n"
            f"p.LIB_PATH = {str(tmp_path / 'missing.so')!r}\n"
            "try:\n    p.PolarCode([1, 0, 1, 0, 1, 1, 0, 0], 0, 0, 2)\n"
            "except ImportError as e:\n    print('import-error', e)\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=root, timeout=120)
    assert out.returncode == 0 and "import-error" in out.stdout, out.stderr[-1000:]


def test_workload_pools_cover_the_batched_mix():
    from paper_1505_01466_gb300 import workloads as WL
    pools = WL.class_pools(pool_frames=4, seed=3)
    assert len(pools) == 125
    shapes = {(p.N, p.L) for p in pools}
    assert {N for N, _ in shapes} == {256, 512, 1024, 2048, 4096} and {L for _, L in shapes} == {2, 4, 8, 16, 32}
    p = pools[7]
    x = p.rows(2, 3, "i8")
    assert x.shape == (3, p.N) and x.dtype == np.int8
    assert np.array_equal(p.rows(5, 1, "f32")[0], p.rows(1, 1, "f32")[0])      # rows wrap around the pool


def _paper_alpha_elems(N, L, V):
    # Sec. IV-E: N channel values shared by all paths plus, per path, one stage
    # of max(2^i, V) values for every i < log2 N
    return N + L * sum(max(1 << i, V) for i in range(N.bit_length() - 1))


def _paper_beta_elems(N, L, V):
    # Sec. IV-F: per path the root stage plus a left and a right copy of every lower stage
    return L * (N + 2 * sum(max(1 << i, V) for i in range(N.bit_length() - 1)))


@pytest.mark.parametrize("dtype,es", [(0, 4), (1, 1)])
@pytest.mark.parametrize("L", [4, 8, 32])
def test_stage_memory_follows_the_paper_accounting(polar, dtype, es, L):
    """Growth of the per-frame memory with N, everything in shared memory.

    Alpha: the paper's count, N + L sum_{i<n} max(2^i, V), with V = 1 and
    without the four lowest stages, which live in registers. Per doubling of N the formula grows by N(1 + L)
    elements, and so must the layout. Beta: bit-packed, one left stage per
    level plus one root row updated in place, so it grows by 2LN + N bits
    where the paper's padded float layout grows by 3LN elements.
    """
    sizes = {}
    for N in (256, 512, 1024):
        fr = I.ga_frozen_mask(N, N // 2, 2.0)
        code = polar.PolarCode(fr, 8, I.CRC8_POLY, L, host_only=True)
        code.set_launch(dtype, 1, 232448, 32)
        code.set_recompute(dtype, 0)
        info = code.info()
        if info["spill_mask"][dtype] or info["scratch_per_frame"][dtype]:
            pytest.skip("does not fit shared memory")
        sizes[N] = info["smem_per_frame"][dtype]
    for N in (256, 512):
        grow = sizes[2 * N] - sizes[N]
        alpha = es * (_paper_alpha_elems(2 * N, L, 16) - _paper_alpha_elems(N, L, 16))
        assert alpha == es * N * (1 + L)
        assert grow == alpha + (2 * L * N + N) // 8
        # the paper's beta layout would need 3LN more elements; bit packing
        # and the in-place root row keep it below that even counted in bytes
        assert (2 * L * N + N) // 8 < _paper_beta_elems(2 * N, L, 16) - _paper_beta_elems(N, L, 16)
    # absolute alpha: the formula without SIMD padding (V = 1) minus the
    # 1 + 2 + 4 + 8 register-held values of stages 0..3 of each path, in bytes
    N = 1024
    fr = I.ga_frozen_mask(N, N // 2, 2.0)
    code = polar.PolarCode(fr, 8, I.CRC8_POLY, L, host_only=True)
    code.set_launch(dtype, 1, 232448, 32)
    code.set_recompute(dtype, 0)
    per_path_tables = 2 * 16 + 2 * 16 + 2 * 4 + 8          # alpha/beta index rows, penalties, survivors
    beta_bytes = L * 4 * (sum(max(1, (1 << j) // 32) for j in range(4, 10)) + N // 32) + N // 8
    expect = es * (_paper_alpha_elems(N, L, 1) - 15 * L) + beta_bytes + L * per_path_tables
    assert code.info()["smem_per_frame"][dtype] == expect


def test_l1_codes_report_their_own_kernel(polar):
    """L = 1 codes run the Fast-SSC kernel: one lane per frame, 32 frames per
    warp, alpha stages and beta rows interleaved over the lanes. By default all
    of it sits in global scratch (coalesced, L1-cached); a shared-memory budget
    per warp takes the beta rows first, then the lowest stages that fit;
    set_launch hands the code to the list kernels."""
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 1, host_only=True)
    below = {4: lambda j: (1 << j) - 1, 1: lambda j: j if j <= 2 else (1 << (j - 2)) + 1}
    beta = 64 * 128                                                 # N / 32 words of 32 lanes

    info = code.info()
    for d, es in ((0, 4), (1, 1)):
        assert info["warps_per_frame"][d] == 1 and info["frames_per_cta"][d] == 256
        assert info["smem_per_frame"][d] == 0
        assert info["scratch_per_frame"][d] == (below[es](11) * 128 + beta) // 32
        assert info["spill_mask"][d] == (1 << 11) - 1
    code.set_smem_budget(0, 48 * 1024)                              # f32: beta rows and stages 0..7
    smem = below[4](8) * 128 + beta
    assert smem <= 48 * 1024 < below[4](9) * 128 + beta
    info = code.info()
    assert info["smem_per_frame"][0] == smem // 32 and info["frames_per_cta"][0] == 32 * min(8, 232448 // smem)
    assert info["scratch_per_frame"][0] == (below[4](11) - below[4](8)) * 128 // 32
    assert info["spill_mask"][0] == ((1 << 11) - 1) & ~0xFF
    code.set_smem_budget(1, 232448)                                 # int8: every stage on chip
    smem = below[1](11) * 128 + beta
    assert code.info()["smem_per_frame"][1] == smem // 32 and code.info()["scratch_per_frame"][1] == 0
    assert code.info()["frames_per_cta"][1] == 32 * (232448 // smem)
    code.set_launch(0, 1, 7000, 512)
    assert code.info()["frames_per_cta"][0] == 16 and code.info()["scratch_per_frame"][0] > 0
    code.set_smem_budget(0, 0)                                      # back to the L = 1 kernel
    assert code.info()["frames_per_cta"][0] == 256
    with pytest.raises(polar.PolarError):
        polar.PolarCode(fr, 32, I.CRC32_POLY, 4, host_only=True).set_smem_budget(0, 0)


def test_recomputed_stages_leave_the_layout(polar):
    """Top stages evaluated from the channel take no memory: at (2048,1723)
    L = 32 (stage 8 holds a Rate-1 leaf, so at most stages 9 and 10
    qualify) depth 2 removes exactly L (1024 + 512) values per frame."""
    fr = I.ga_frozen_mask(2048, 1723, 4.0, 1691 / 2048)
    code = polar.PolarCode(fr, 32, I.CRC32_POLY, 32, host_only=True)
    info = code.info()
    assert info["max_recompute_depth"] == 2
    assert info["recomputed_stages"] == [0, 0]                    # every stage stored by default
    for dt, es in ((0, 4), (1, 1)):
        code.set_launch(dt, 1, 7000, 512)
        code.set_recompute(dt, 0)
        full = code.info()["scratch_per_frame"][dt]
        code.set_recompute(dt, 2)
        assert code.info()["recomputed_stages"][dt] == 0x600
        assert full - code.info()["scratch_per_frame"][dt] == 32 * (1024 + 512) * es
        with pytest.raises(polar.PolarError):
            code.set_recompute(dt, 3)
    # a code whose top stage holds a leaf has nothing to evaluate
    half = np.zeros(1024, np.uint8)
    half[:512] = 1                                                 # left half Rate-0, right half Rate-1
    c2 = polar.PolarCode(half, 0, 0, 8, host_only=True)
    assert c2.info()["max_recompute_depth"] == 0 and c2.info()["recomputed_stages"] == [0, 0]


def test_packing_needs_a_packable_shape(polar):
    fr = I.ga_frozen_mask(1024, 860, 4.0, 828 / 1024)
    c8 = polar.PolarCode(fr, 32, I.CRC32_POLY, 8, host_only=True)
    c8.set_launch(0, 1, 7000, 128)                 # 4 frame groups per CTA: 32 / 8 = 4 frames to a warp
    c8.set_packing(0, True)
    c8.set_packing(0, False)
    c8.set_launch(0, 2, 7000, 128)                 # two warps per frame: no packing
    with pytest.raises(polar.PolarError):
        c8.set_packing(0, True)
    c4 = polar.PolarCode(fr, 32, I.CRC32_POLY, 4, host_only=True)
    c4.set_launch(1, 1, 7000, 128)                 # 8 frames to a warp need 8 groups per CTA:
    c4.set_packing(1, True)                        # segments alone
    assert c4.info()["packed"][1] == 1
    c4.set_launch(1, 1, 7000, 256)
    c4.set_packing(1, True)
    c32 = polar.PolarCode(fr, 32, I.CRC32_POLY, 32, host_only=True)
    with pytest.raises(polar.PolarError):
        c32.set_packing(0, True)


def test_packing_default_and_choice_follow_the_code(polar):
    """Packing is on by default for L <= 4 and off for L = 8, 16; a choice made
    with set_packing is kept by later one-warp shapes and dropped by shapes
    with more warps per frame."""
    fr = I.ga_frozen_mask(1024, 860, 4.0, 828 / 1024)
    for L, default in ((2, 1), (4, 1), (8, 0), (16, 0), (32, 0)):
        c = polar.PolarCode(fr, 32, I.CRC32_POLY, L, host_only=True)
        c.set_launch(1, 1, 7000, 512)
        assert c.info()["packed"][1] == default, L
        c.set_launch(1, 2, 7000, 512)
        assert c.info()["packed"][1] == 0, L
    c8 = polar.PolarCode(fr, 32, I.CRC32_POLY, 8, host_only=True)
    c8.set_launch(0, 1, 7000, 512)
    c8.set_packing(0, True)
    c8.set_launch(0, 1, 14000, 256)                # the choice outlives the shape
    assert c8.info()["packed"] == [1, 0]
    c8.set_launch(0, 4, 14000, 256)
    assert c8.info()["packed"][0] == 0
    c8.set_launch(0, 1, 7000, 512)                 # and comes back with one warp per frame
    assert c8.info()["packed"][0] == 1
    c2 = polar.PolarCode(fr, 32, I.CRC32_POLY, 2, host_only=True)
    c2.set_launch(0, 1, 7000, 512)
    c2.set_packing(0, False)
    c2.set_launch(0, 1, 7000, 256)
    assert c2.info()["packed"][0] == 0
