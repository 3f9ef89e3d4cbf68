"""GPU tests of the batched form: frames of several codes in one persistent
launch must give exactly what the plain decoder gives for each frame (and so
what the oracle gives), including through a captured CUDA graph."""
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
    import paper_1505_01466_gb300.polar as polar
    return torch, polar


CLASSES = [(256, 64, 2), (512, 256, 8), (1024, 860, 32), (2048, 1723, 8), (256, 230, 16), (4096, 3686, 4),
           (128, 64, 1)]


def _mixed(polar, dtype, n_frames, seed):
    codes, frozen, frames = [], [], []
    rng = np.random.default_rng(seed)
    fc = rng.integers(0, len(CLASSES), n_frames).astype(np.uint32)
    per_class = []
    for c, (N, K, L) in enumerate(CLASSES):
        fr = I.ga_frozen_mask(N, K, 4.0, (K - 32) / N)
        frozen.append(fr)
        codes.append(polar.PolarCode(fr, 32, I.CRC32_POLY, L))
        cnt = int((fc == c).sum())
        f = I.make_frames(fr, 32, I.CRC32_POLY, float(rng.uniform(1.0, 4.0)), max(cnt, 1), seed=seed * 100 + c)
        per_class.append(f.llr_i8 if dtype == "i8" else f.llr_f32)
    idx = np.zeros(len(CLASSES), np.int64)
    rows = []
    for f in range(n_frames):
        c = fc[f]
        rows.append(per_class[c][idx[c]])
        idx[c] += 1
    return codes, frozen, fc, rows


def _run_batch(torch, polar, codes, fc, rows, dtype, graph=False, tune=False, launch=None):
    dt = polar.LLR_I8 if dtype == "i8" else polar.LLR_F32
    b = polar.PolarBatch(codes, fc, dt)
    llr_bytes, bits_bytes, lo, bo = b.layout()
    packed = np.concatenate([r.view(np.uint8).ravel() for r in rows])
    assert packed.size == llr_bytes and np.array_equal(lo[1:], np.cumsum([r.nbytes for r in rows])[:-1])
    llr = torch.from_numpy(packed).cuda()
    F = len(rows)
    bits = torch.zeros(bits_bytes, dtype=torch.uint8, device="cuda")
    pm = torch.zeros(F, dtype=torch.float32, device="cuda")
    ok = torch.zeros(F, dtype=torch.uint8, device="cuda")
    slot = torch.zeros(F, dtype=torch.int32, device="cuda")
    if launch is not None:
        b.set_launch(*launch)
    if tune:
        b.autotune(llr, bits, pm)
    if graph:
        s = torch.cuda.Stream()
        b.capture(llr, bits, pm, ok, slot, stream=s)
        bits.zero_(); pm.zero_(); ok.zero_(); slot.fill_(-1)
        b.replay(stream=s)
        b.replay(stream=s)
        s.synchronize()
    else:
        b.run(llr, bits, pm, ok, slot)
    torch.cuda.synchronize()
    out = (bits.cpu().numpy(), pm.cpu().numpy(), ok.cpu().numpy(), slot.cpu().numpy(), bo)
    b.close()
    return out


def _check_against_plain(torch, codes, fc, rows, out):
    bits, pm, ok, slot, bo = out
    for c, code in enumerate(codes):
        sel = np.flatnonzero(fc == c)
        if sel.size == 0:
            continue
        llr = torch.from_numpy(np.stack([rows[i] for i in sel])).cuda()
        gb, gpm, gok, gsl = (t.cpu().numpy() for t in code.decode(llr))
        kb = (code.k + 7) // 8
        for j, i in enumerate(sel):
            assert np.array_equal(bits[int(bo[i]): int(bo[i]) + kb], gb[j]), (c, i)
        assert np.array_equal(pm[sel], gpm) and np.array_equal(ok[sel], gok) and np.array_equal(slot[sel], gsl)


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_batch_equals_plain_and_oracle(env, oracle_mod, dtype):
    torch, polar = env
    codes, frozen, fc, rows = _mixed(polar, dtype, 700, seed=3)
    out = _run_batch(torch, polar, codes, fc, rows, dtype)
    _check_against_plain(torch, codes, fc, rows, out)
    bits, pm, ok, slot, bo = out
    # a sample of frames against the oracle
    for c, (N, K, L) in enumerate(CLASSES):
        sel = np.flatnonzero(fc == c)[:6]
        if sel.size == 0:
            continue
        ob, opm, ook, osl = oracle_mod.decode(frozen[c], L, np.stack([rows[i] for i in sel]), 32, I.CRC32_POLY,
                                              0, n_threads=NT)
        kb = (K - 32 + 7) // 8
        for j, i in enumerate(sel):
            assert np.array_equal(bits[int(bo[i]): int(bo[i]) + kb], ob[j])
        assert np.array_equal(slot[sel], osl) and np.array_equal(ok[sel], ook)
        np.testing.assert_allclose(pm[sel], opm, rtol=1e-5, atol=0)


def test_batch_graph_replay_and_autotune(env):
    torch, polar = env
    codes, frozen, fc, rows = _mixed(polar, "i8", 500, seed=4)
    ref = _run_batch(torch, polar, codes, fc, rows, "i8")
    for graph, tune in ((True, False), (False, True), (True, True)):
        out = _run_batch(torch, polar, codes, fc, rows, "i8", graph=graph, tune=tune)
        for a, b in zip(out, ref):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("launch", [(1, 7000, 512), (1, 0, 256), (2, 20000, 256), (4, 0, 512)])
def test_batch_cta_sizes_and_lockstep_units(env, launch):
    # CTAs of several groups: units whose frames share a code run in lockstep,
    # mixed units (class boundaries, the ragged end) run without it
    torch, polar = env
    codes, frozen, fc, rows = _mixed(polar, "i8", 613, seed=6)
    ref = _run_batch(torch, polar, codes, fc, rows, "i8")
    out = _run_batch(torch, polar, codes, fc, rows, "i8", launch=launch)
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)
