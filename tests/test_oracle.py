"""Pins for the CPU oracle (CPU only).

The oracle is checked against things that do not come from it:

* brute-force maximum likelihood: with L >= 2^K nothing is pruned, so the
  final list of the SC-list decoder holds every codeword, and with min-sum
  (max-log) updates each path's penalty telescopes to the correlation
  discrepancy sum_{i: x_i != h(y_i)} |y_i| (Eq. (6) summed down the tree);
  the fast decoder must give the same list when its nodes are exhaustive
  (Rate-1 of length <= 2, SPC of length 4, repetition, Rate-0);
* noiseless frames decode to the sent payload with penalty 0;
* the (8,4) example of Fig. 1 / Fig. 2 / Listing 2;
* codes whose forking leaves each carry a single information bit make the
  fast decoder and bit-by-bit SC-list take identical decisions at any L;
* the fast decoder's frame-error rate matches SC-list (Sec. VI) within
  Monte-Carlo confidence;
* the final pick (Sec. II-B) recomputed outside the oracle from its final
  list: u = x G_N, the CRC from ``inputs``, the least (penalty, slot) among
  the passing paths, on frames where a lower-penalty path fails the CRC;
* int8 G saturation at +-127 on a (4,2) example worked by hand;
* pruned selection (2 <= L < 2^K) against an independently written
  bit-by-bit SC-list that recomputes every LLR from the channel;
* plausible single mistakes planted in a copy of the oracle source fail at
  least one of these checks.
"""
import itertools
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1505_01466_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def _brute_force(frozen, y):
    """All codewords with their correlation discrepancy penalties."""
    N = frozen.size
    info = np.flatnonzero(frozen == 0)
    hy = (y < 0).astype(np.uint8)
    out = []
    for bits in itertools.product((0, 1), repeat=info.size):
        u = np.zeros(N, np.uint8)
        u[info] = bits
        x = I.polar_transform(u)
        out.append((float(np.abs(y[x != hy]).sum()), tuple(int(v) for v in x)))
    return sorted(out)


def _final_list(oracle_mod, frozen, L, y, mode):
    words, pens = oracle_mod.decode_list(frozen, L, y, mode)
    return sorted((float(p), tuple(int(v) for v in w)) for w, p in zip(words, pens))


def _random_code(rng, N, K):
    fr = np.ones(N, np.uint8)
    fr[rng.choice(N, K, replace=False)] = 0
    return fr


def _fast_leaves_exhaustive(oracle_mod, frozen, mode):
    for kind, nv, _ in oracle_mod.schedule(frozen, mode):
        if kind == oracle_mod.LEAF_RATE1 and nv > 2:
            return False
        if kind == oracle_mod.LEAF_SPC and nv != 4:
            return False
    return True


def test_golden_fig1_schedule(oracle_mod):
    names = {"F": 0, "G": 1, "COMBINE": 2, "RATE0": 11, "RATE1": 12, "REP": 13, "SPC": 14}
    frozen, info, ops = None, None, []
    with open(os.path.join(HERE, "golden", "fig1_code_8_4.txt")) as fh:
        for line in fh:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "frozen":
                frozen = np.array([int(v) for v in t[1:]], np.uint8)
            elif t[0] == "info":
                info = [int(v) for v in t[1:]]
            elif t[0] == "op":
                ops.append((names[t[1]], int(t[2]), int(t[3])))
    assert list(np.flatnonzero(frozen == 0)) == info
    assert oracle_mod.schedule(frozen, oracle_mod.SPC4) == ops
    # the information set also comes out of the GA construction (Fig. 1)
    assert np.array_equal(I.ga_frozen_mask(8, 4, 2.0), frozen)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_scl_list_equals_brute_force_ml(oracle_mod, dtype):
    rng = np.random.default_rng(11)
    for trial in range(40):
        N = int(rng.choice([4, 8, 16]))
        K = int(rng.integers(1, min(N, 6) + 1))
        fr = _random_code(rng, N, K)
        L = 1 << K
        y = rng.integers(-6, 7, N).astype(np.float32)
        yy = y.astype(np.int8) if dtype == "i8" else y
        bf = _brute_force(fr, y)
        assert _final_list(oracle_mod, fr, L, yy, oracle_mod.BITWISE) == bf
        # the winner (no CRC) is a maximum-likelihood codeword
        _, pm, ok, _ = oracle_mod.decode(fr, L, yy[None], 0, 0, oracle_mod.BITWISE)
        assert pm[0] == bf[0][0] and ok[0] == 1


@pytest.mark.parametrize("mode", ["SPC4", "SPC_ANY"])
def test_fast_list_equals_brute_force_when_nodes_exhaustive(oracle_mod, mode):
    m = getattr(oracle_mod, mode)
    rng = np.random.default_rng(12)
    checked = 0
    while checked < 40:
        N = int(rng.choice([4, 8, 16, 32]))
        K = int(rng.integers(1, min(N, 7) + 1))
        fr = _random_code(rng, N, K)
        if not _fast_leaves_exhaustive(oracle_mod, fr, m):
            continue
        y = rng.integers(-7, 8, N).astype(np.float32)
        assert _final_list(oracle_mod, fr, 1 << K, y, m) == _brute_force(fr, y)
        checked += 1


def test_fast_nonexhaustive_rate1_keeps_the_ml_word(oracle_mod):
    # A Rate-1 node of length 8 (two least-reliable-bit Chase search) still
    # puts the hard decision, i.e. the ML word of the node, on the list.
    fr = np.zeros(8, np.uint8)
    rng = np.random.default_rng(3)
    for _ in range(20):
        y = rng.integers(-9, 10, 8).astype(np.float32)
        words, pens = oracle_mod.decode_list(fr, 4, y, oracle_mod.SPC4)
        assert len(words) == 4
        assert np.array_equal(words[np.argmin(pens)], (y < 0).astype(np.uint8))
        assert pens.min() == 0.0


@pytest.mark.parametrize("dtype", ["f32", "i8"])
@pytest.mark.parametrize("mode", ["BITWISE", "SPC4", "SPC_ANY"])
def test_noiseless_decodes_sent_payload(oracle_mod, dtype, mode):
    fr = I.ga_frozen_mask(256, 128, 2.0, 120 / 256)
    f = I.make_frames(fr, 8, I.CRC8_POLY, 2.0, 12, seed=7, noiseless=True)
    llr = f.llr_i8 if dtype == "i8" else f.llr_f32
    for L in (1, 2, 4, 8):
        bits, pm, ok, slot = oracle_mod.decode(fr, L, llr, 8, I.CRC8_POLY, getattr(oracle_mod, mode))
        assert np.array_equal(I.unpack_bits_lsb(bits, 120), f.payload)
        assert (pm == 0).all() and (ok == 1).all()


def _sc_decode(frozen, y):
    """Textbook recursive successive-cancellation decoder (min-sum)."""
    def rec(a, fr):
        if a.size == 1:
            return np.array([0 if fr[0] else int(a[0] < 0)], np.uint8)
        h = a.size // 2
        l, r = a[:h], a[h:]
        fa = np.sign(l) * np.sign(r) * np.minimum(np.abs(l), np.abs(r))
        bl = rec(fa.astype(np.float32), fr[:h])
        ga = (r + (1 - 2 * bl.astype(np.float32)) * l).astype(np.float32)
        br = rec(ga, fr[h:])
        return np.concatenate([bl ^ br, br])
    return rec(np.asarray(y, np.float32), frozen)


def test_scl_with_one_path_is_sc(oracle_mod):
    fr = I.ga_frozen_mask(64, 32, 1.0)
    f = I.make_frames(fr, 0, 0, 1.0, 60, seed=21)
    bits, _, _, _ = oracle_mod.decode(fr, 1, f.llr_f32, 0, 0, oracle_mod.BITWISE)
    info = I.info_positions(fr)
    for i in range(60):
        x = _sc_decode(fr, f.llr_f32[i])
        u = I.polar_transform(x)
        assert np.array_equal(I.unpack_bits_lsb(bits[i], 32), u[info])


def _single_info_leaf_code(rng, N):
    """Random frozen set whose Fast-SSC leaves are Rate-0, repetition or one-bit Rate-1."""
    def rec(n):
        r = rng.random()
        if n == 1:
            return [int(rng.random() < 0.45)]  # 1 = frozen
        if r < 0.2:
            return [1] * n
        if r < 0.45:
            return [1] * (n - 1) + [0]
        return rec(n // 2) + rec(n // 2)
    return np.array(rec(N), np.uint8)


def test_fast_equals_scl_when_each_fork_has_one_info_bit(oracle_mod):
    rng = np.random.default_rng(4)
    checked = 0
    while checked < 25:
        N = int(rng.choice([16, 32, 64]))
        fr = _single_info_leaf_code(rng, N)
        sch = oracle_mod.schedule(fr, oracle_mod.SPC4)
        if any(k == oracle_mod.LEAF_RATE1 and nv > 1 for k, nv, _ in sch) or \
           any(k == oracle_mod.LEAF_SPC for k, _, _ in sch) or (fr == 0).sum() == 0:
            continue
        y = rng.integers(-8, 9, (6, N)).astype(np.float32)
        for L in (1, 2, 4, 8):
            a = oracle_mod.decode(fr, L, y, 0, 0, oracle_mod.BITWISE)
            b = oracle_mod.decode(fr, L, y, 0, 0, oracle_mod.SPC4)
            for u, v in zip(a, b):
                assert np.array_equal(u, v)
            for i in range(6):
                wa, pa = oracle_mod.decode_list(fr, L, y[i], oracle_mod.BITWISE)
                wb, pb = oracle_mod.decode_list(fr, L, y[i], oracle_mod.SPC4)
                assert np.array_equal(wa, wb) and np.array_equal(pa, pb)
        checked += 1


def _two_proportion_ok(e1, e2, n, z=2.576):
    p = (e1 + e2) / (2 * n)
    if p == 0:
        return True
    se = math.sqrt(2 * p * (1 - p) / n)
    return abs(e1 - e2) / n <= z * se + 1.0 / n


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_fast_fer_matches_scl(oracle_mod, dtype):
    # Sec. VI: Dec-SPC-4 matches the SC-list error-correction performance.
    fr = I.ga_frozen_mask(256, 128, 2.0, 120 / 256)
    f = I.make_frames(fr, 8, I.CRC8_POLY, 1.75, 2000, seed=2024)
    llr = f.llr_i8 if dtype == "i8" else f.llr_f32
    errs = {}
    for mode in (oracle_mod.BITWISE, oracle_mod.SPC4):
        bits, _, _, _ = oracle_mod.decode(fr, 4, llr, 8, I.CRC8_POLY, mode, n_threads=8)
        errs[mode] = int((I.unpack_bits_lsb(bits, 120) != f.payload).any(1).sum())
    assert errs[oracle_mod.BITWISE] >= 20          # enough errors to be meaningful
    assert _two_proportion_ok(errs[oracle_mod.BITWISE], errs[oracle_mod.SPC4], 2000), errs


# ---------------------------------------------------------------------------
# Final pick (Sec. II-B): the output is the best path that passes the CRC.
# ---------------------------------------------------------------------------
def _crc_first_pick(frozen, crc_len, poly, words, pens):
    """Winner of a final list, recomputed outside the oracle: u = x G_N, the
    information bits in ascending index, the payload/CRC split and the CRC
    from ``inputs``; the least (penalty, slot) among the passing paths, else
    among all paths. Returns (slot, crc_ok, payload bits)."""
    info = I.info_positions(frozen)
    k = info.size - crc_len
    u = I.polar_transform(np.asarray(words, np.uint8))[:, info]
    ok = (I.crc_bits(u[:, :k], crc_len, poly) == u[:, k:]).all(axis=1)
    order = np.lexsort((np.arange(len(pens)), np.asarray(pens)))   # by (penalty, slot)
    passing = [s for s in order if ok[s]]
    s = int(passing[0] if passing else order[0])
    return s, int(ok[s]), u[s, :k]


def _crc_first_frames(mod, N, K, L, ebn0, n, seed, dtype="f32", mode=None):
    """Noisy frames whose least-penalty final path fails the CRC while
    another path passes it: (frozen, llr [F, N], expected picks)."""
    mode = mod.SPC4 if mode is None else mode
    fr = I.ga_frozen_mask(N, K, 2.0, (K - 8) / N)
    f = I.make_frames(fr, 8, I.CRC8_POLY, ebn0, n, seed=seed)
    llr = f.llr_i8 if dtype == "i8" else f.llr_f32
    rows, want = [], []
    for i in range(n):
        words, pens = mod.decode_list(fr, L, llr[i], mode)
        s, ok, payload = _crc_first_pick(fr, 8, I.CRC8_POLY, words, pens)
        least = int(np.lexsort((np.arange(len(pens)), pens))[0])
        if ok and s != least:
            rows.append(i)
            want.append((s, float(pens[s]), payload))
    return fr, llr[rows], want


@pytest.mark.parametrize("N,K,L,ebn0,dtype", [(64, 40, 8, 1.0, "f32"), (64, 40, 4, 1.0, "i8"),
                                              (256, 128, 8, 1.0, "f32"), (256, 128, 4, 1.0, "i8")])
def test_final_pick_prefers_crc_passing_path(oracle_mod, N, K, L, ebn0, dtype):
    fr, llr, want = _crc_first_frames(oracle_mod, N, K, L, ebn0, 300, seed=77 + N + L, dtype=dtype)
    assert len(want) >= 20, len(want)       # frames where the rule decides the output
    bits, pm, ok, slot = oracle_mod.decode(fr, L, llr, 8, I.CRC8_POLY, oracle_mod.SPC4)
    for i, (s, pen, payload) in enumerate(want):
        assert slot[i] == s and ok[i] == 1 and pm[i] == pen
        assert np.array_equal(I.unpack_bits_lsb(bits[i], K - 8), payload)


def test_final_pick_falls_back_to_least_penalty(oracle_mod):
    # a CRC that no path passes: every word's CRC bits are forced wrong by
    # decoding against a different polynomial than the frames were built with
    fr = I.ga_frozen_mask(64, 40, 2.0, 32 / 64)
    f = I.make_frames(fr, 8, I.CRC8_POLY, 1.0, 40, seed=5)
    bits, pm, ok, slot = oracle_mod.decode(fr, 4, f.llr_f32, 8, 0x9B, oracle_mod.SPC4)
    for i in range(40):
        words, pens = oracle_mod.decode_list(fr, 4, f.llr_f32[i], oracle_mod.SPC4)
        s, okk, payload = _crc_first_pick(fr, 8, 0x9B, words, pens)
        assert slot[i] == s and ok[i] == okk and pm[i] == pens[s]
        assert np.array_equal(I.unpack_bits_lsb(bits[i], 32), payload)


# ---------------------------------------------------------------------------
# int8 G saturates at +-127 (the int8 convention; the paper is float-only).
# ---------------------------------------------------------------------------
# A (4,2) code with u0 and u2 frozen, decoded bit by bit with L = 4 so every
# codeword stays on the list. Worked by hand from Eqs. (1)-(3) and Eq. (6):
#
#   y = (100, 100, 100, 100):
#     F at the root: (f(100,100), f(100,100)) = (100, 100); u0: f(100,100)
#     = 100, frozen, h = 0, no penalty. u1: G = 100 + 100 = 200 -> 127 in int8.
#     Slots (s, c) order: A = (u1 = 0, P = 0), B = (u1 = 1, P = 127 | 200).
#     G at the root with beta_left = (u0^u1, u1): A gets (200, 200) -> (127,
#     127); B gets (0, 0). u2 frozen: A f(127,127) = 127, B f(0,0) = 0: no
#     penalty. u3: A lambda = 127 + 127 -> 127 (f32: 400), B lambda = 0.
#     Final slots (A,0) (A,1) (B,0) (B,1), words x = uG:
#       0000 P 0; 1111 P 127 | 400; 1100 P 127 | 200; 0011 P 127 | 200.
#   y = (100, -100, 100, -100):
#     the same up to the root's G, which gives A (200, -200) -> (127, -127)
#     and B (0, 0). u2 frozen: A f(127, -127) = -127, h = 1, P += 127 | 200;
#     B: 0. u3: A lambda = -127 + 127 = 0 (f32: -200 + 200 = 0), B lambda = 0.
#     Final: every slot P = 127 (int8) | 200 (f32), the same four words.
# The f32 penalties equal each word's correlation discrepancy (100 x the
# positions where x differs from h(y)); int8 caps every G at 127.
SAT_CASES = [
    ((100, 100, 100, 100), [0, 127, 127, 127], [0, 400, 200, 200]),
    ((100, -100, 100, -100), [127, 127, 127, 127], [200, 200, 200, 200]),
]
SAT_WORDS = [(0, 0, 0, 0), (1, 1, 1, 1), (1, 1, 0, 0), (0, 0, 1, 1)]


def _saturation_pins(mod):
    fr = np.array([1, 0, 1, 0], np.uint8)
    for y, pen_i8, pen_f32 in SAT_CASES:
        for arr, want in ((np.array(y, np.int8), pen_i8), (np.array(y, np.float32), pen_f32)):
            words, pens = mod.decode_list(fr, 4, arr, mod.BITWISE)
            if [tuple(int(v) for v in w) for w in words] != SAT_WORDS:
                return False
            if [float(p) for p in pens] != [float(v) for v in want]:
                return False
    return True


def test_int8_g_saturates_hand_worked(oracle_mod):
    assert _saturation_pins(oracle_mod)


def test_int8_fast_nodes_see_saturated_llrs(oracle_mod):
    # The same frames through the fast node rules: the root of the (4,2) code
    # splits into two repetition nodes of length 2; the right one sees the
    # saturated G outputs, so its repetition penalties are sums of +-127.
    fr = np.array([1, 0, 1, 0], np.uint8)
    words, pens = oracle_mod.decode_list(fr, 4, np.array((100, 100, 100, 100), np.int8), oracle_mod.SPC4)
    got = sorted((float(p), tuple(int(v) for v in w)) for w, p in zip(words, pens))
    # left rep node: alpha = (100, 100): P0 = 0, P1 = 200 (sums of the inputs
    # themselves, no G). Right node: path u1 = 0 sees (127, 127) -> P0 = 0,
    # P1 = 254; path u1 = 1 sees (0, 0) -> 0 and 0.
    assert got == sorted([(0.0, (0, 0, 0, 0)), (254.0, (1, 1, 1, 1)),
                          (200.0, (1, 1, 0, 0)), (200.0, (0, 0, 1, 1))])


# ---------------------------------------------------------------------------
# Pruned selection (Algorithm 1 with 2 <= L < 2^K): an independent SC-list.
# ---------------------------------------------------------------------------
def _py_scl(frozen, y, L, sat):
    """Bit-by-bit LLR SC-list, written independently of the oracle: the LLR
    of bit i is recomputed from the channel for every path by the recursion
    on the halves of the code (left half: F of the two halves; right half:
    G with the re-encoded left half), the metric follows Eq. (6), and the L
    best of (penalty, source, candidate) survive in (source, candidate)
    order. Integer-valued inputs, so every sum is exact."""
    def clamp(v):
        return max(-127, min(127, v)) if sat else v

    def lam(a, u, i):
        if len(a) == 1:
            return a[0]
        h = len(a) // 2
        if i < h:
            fa = [(1 if (a[t] < 0) == (a[t + h] < 0) else -1) * min(abs(a[t]), abs(a[t + h]))
                  for t in range(h)]
            return lam(fa, u, i)
        bl = I.polar_transform(np.array(u[:h], np.uint8))
        ga = [clamp(a[t + h] + (1 - 2 * int(bl[t])) * a[t]) for t in range(h)]
        return lam(ga, u[h:], i - h)

    y = [max(-127, int(v)) if sat else int(v) for v in y]
    paths = [(0, [])]
    for i in range(len(y)):
        if frozen[i]:
            new = []
            for pen, u in paths:
                v = lam(y, u, i)
                new.append((pen + (abs(v) if v < 0 else 0), u + [0]))
            paths = new
            continue
        cands = []
        for s, (pen, u) in enumerate(paths):
            v = lam(y, u, i)
            hd = 1 if v < 0 else 0
            cands.append((pen, s, 0, u + [hd]))
            cands.append((pen + abs(v), s, 1, u + [1 - hd]))
        keep = sorted(cands, key=lambda c: (c[0], c[1], c[2]))[:L]
        keep.sort(key=lambda c: (c[1], c[2]))
        paths = [(c[0], c[3]) for c in keep]
    return [(float(p), tuple(int(b) for b in I.polar_transform(np.array(u, np.uint8)))) for p, u in paths]


def _pruned_selection_pins(mod, trials, seed):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        N = int(rng.choice([8, 16, 32]))
        K = int(rng.integers(3, min(N, 10) + 1))
        fr = _random_code(rng, N, K)
        for L in (2, 4):
            if L >= (1 << K):
                continue
            sat = bool(rng.integers(0, 2))
            if sat:
                y = rng.integers(-127, 128, N).astype(np.int8)
            else:
                y = rng.integers(-8, 9, N).astype(np.float32)
            words, pens = mod.decode_list(fr, L, y, mod.BITWISE)
            got = [(float(p), tuple(int(v) for v in w)) for w, p in zip(words, pens)]
            if got != _py_scl(fr, y, L, sat):
                return False
    return True


def test_pruned_selection_equals_independent_scl(oracle_mod):
    assert _pruned_selection_pins(oracle_mod, 60, 31)


# ---------------------------------------------------------------------------
# Planted mistakes: each textual mutation of the oracle must fail a pin.
# ---------------------------------------------------------------------------
MUTATIONS = [
    ("G sign", "float r = beta ? b - a : b + a;", "float r = beta ? b + a : b - a;"),
    ("F uses max", "float m = ma < mb ? ma : mb;", "float m = ma > mb ? ma : mb;"),
    ("F drops sign", "return ((a < 0.0f) != (b < 0.0f)) ? -m : m;", "return m;"),
    ("Rate-0 uses max", "for (int i = 0; i < nv; ++i) t[i] = a[i] < 0.0f ? -a[i] : 0.0f;",
     "for (int i = 0; i < nv; ++i) t[i] = a[i] > 0.0f ? a[i] : 0.0f;"),
    ("combine direction", "for (int i = 0; i < h; ++i) b[i] ^= b[i + h];",
     "for (int i = 0; i < h; ++i) b[i + h] ^= b[i];"),
    ("SPC parity inverted", "int q = parity == 0;", "int q = parity != 0;"),
    ("Rate-1 flips wrong bit", "ocand_t c1 = {s, 1, pen_s + a1, 0, 1, {m[0], 0, 0, 0}};",
     "ocand_t c1 = {s, 1, pen_s + a1, 0, 1, {m[1], 0, 0, 0}};"),
    ("REP penalties swapped", "float p0 = tree_sum(t0, nv), p1 = tree_sum(t1, nv);",
     "float p1 = tree_sum(t0, nv), p0 = tree_sum(t1, nv);"),
    ("selection keeps worst", "if (x->pen < y->pen) return -1;", "if (x->pen < y->pen) return 1;"),
    ("h of zero", "static int h_of(float a) { return a < 0.0f ? 1 : 0; }",
     "static int h_of(float a) { return a <= 0.0f ? 1 : 0; }"),
    ("final pick ignores CRC", "else if (ok != best.ok) better = ok > best.ok;",
     "else if (0) better = ok > best.ok;"),
    ("G unsaturated", "    if (sat) {\n        if (r > 127.0f)", "    if (0) {\n        if (r > 127.0f)"),
    ("G saturates one side", "if (r < -127.0f) r = -127.0f;", "if (r < -128.0f) r = -128.0f;"),
    ("survivors in key order", "    int slot = 0;\n    for (int i = 0; i < nc; ++i) {",
     "    memcpy(cand, sorted, sizeof(ocand_t) * (size_t)nc);\n    memset(survive, 0, (size_t)nc);\n"
     "    memset(survive, 1, (size_t)keep);\n    int slot = 0;\n    for (int i = 0; i < nc; ++i) {"),
]


def _pins_pass(mod):
    """A compact run of the pins above against an oracle module."""
    rng = np.random.default_rng(99)
    for _ in range(30):
        N = int(rng.choice([4, 8, 16]))
        K = int(rng.integers(1, min(N, 5) + 1))
        fr = _random_code(rng, N, K)
        y = rng.integers(-6, 7, N).astype(np.float32)
        if _final_list(mod, fr, 1 << K, y, mod.BITWISE) != _brute_force(fr, y):
            return False
        if _fast_leaves_exhaustive(mod, fr, mod.SPC4):
            if _final_list(mod, fr, 1 << K, y, mod.SPC4) != _brute_force(fr, y):
                return False
    # zero LLRs: h(0) = 0, so the all-zero word has penalty 0
    fr = I.ga_frozen_mask(16, 8, 2.0)
    w, p = mod.decode_list(fr, 1, np.zeros(16, np.float32), mod.SPC4)
    if p[0] != 0 or w[0].any():
        return False
    fr = I.ga_frozen_mask(64, 40, 3.0)
    f = I.make_frames(fr, 8, I.CRC8_POLY, 3.0, 4, seed=5, noiseless=True)
    for mode in (mod.BITWISE, mod.SPC4):
        bits, pm, ok, _ = mod.decode(fr, 4, f.llr_f32, 8, I.CRC8_POLY, mode)
        if not np.array_equal(I.unpack_bits_lsb(bits, 32), f.payload) or pm.any():
            return False
    # the CRC decides the final pick over a lower penalty (Sec. II-B)
    fr, llr, want = _crc_first_frames(mod, 64, 40, 8, 1.0, 120, seed=149)
    if len(want) < 5:
        return False
    bits, pm, ok, slot = mod.decode(fr, 8, llr, 8, I.CRC8_POLY, mod.SPC4)
    for i, (s, pen, payload) in enumerate(want):
        if slot[i] != s or ok[i] != 1 or pm[i] != pen:
            return False
        if not np.array_equal(I.unpack_bits_lsb(bits[i], 32), payload):
            return False
    # int8 G saturation, worked by hand; pruned selection against an independent SC-list
    return _saturation_pins(mod) and _pruned_selection_pins(mod, 12, 5)


def test_pins_pass_on_the_oracle(oracle_mod):
    assert _pins_pass(oracle_mod)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    import importlib.util
    src_dir = os.path.join(os.path.dirname(HERE), "oracle")
    dst = tmp_path / "oracle_mut"
    shutil.copytree(src_dir, dst, ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    c_file = dst / "polar_oracle.c"
    text = c_file.read_text()
    assert text.count(old) == 1, name
    c_file.write_text(text.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle_mut", dst / "__init__.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(force=True)
    assert not _pins_pass(mod), f"mutation '{name}' was not detected"


def test_adaptive_decoder_properties(oracle_mod):
    # Sec. V: Fast-SSC first, the list decoder only where the CRC failed.
    fr = I.ga_frozen_mask(256, 128, 2.0, 120 / 256)
    clean = I.make_frames(fr, 8, I.CRC8_POLY, 2.0, 16, seed=3, noiseless=True)
    b, pm, ok, slot, n = oracle_mod.adaptive_decode(fr, 8, clean.llr_f32, 8, I.CRC8_POLY)
    assert n == 0 and ok.all() and np.array_equal(I.unpack_bits_lsb(b, 120), clean.payload)
    f = I.make_frames(fr, 8, I.CRC8_POLY, 1.5, 400, seed=4)
    b, pm, ok, slot, n = oracle_mod.adaptive_decode(fr, 8, f.llr_f32, 8, I.CRC8_POLY)
    _, _, ok1, _ = oracle_mod.decode(fr, 1, f.llr_f32, 8, I.CRC8_POLY)
    _, _, ok8, _ = oracle_mod.decode(fr, 8, f.llr_f32, 8, I.CRC8_POLY)
    assert 0 < n == int((ok1 == 0).sum()) < 400          # both branches taken
    assert np.array_equal(ok, ok1 | ok8)                  # the switch only ever helps
    # a frame whose payload the list decoder gets right is right after the switch too
    right8 = (I.unpack_bits_lsb(oracle_mod.decode(fr, 8, f.llr_f32, 8, I.CRC8_POLY)[0], 120) ==
              f.payload).all(axis=1)
    right = (I.unpack_bits_lsb(b, 120) == f.payload).all(axis=1)
    assert (right | ~right8 | (ok1 == 1)).all()


@pytest.mark.parametrize("mode", ["SPC4", "BITWISE"])
def test_systematic_mode(oracle_mod, mode):
    # noiseless systematic frames decode to their payload; a non-systematic
    # decoder of the same frames finds the same codeword, whose u is not the payload
    fr = I.ga_frozen_mask(256, 128, 2.0, 96 / 256)
    m = getattr(oracle_mod, mode)
    clean = I.make_frames(fr, 32, I.CRC32_POLY, 2.0, 8, seed=2, noiseless=True, systematic=True)
    b, pm, ok, _ = oracle_mod.decode(fr, 4, clean.llr_f32, 32, I.CRC32_POLY, m | oracle_mod.SYSTEMATIC)
    assert ok.all() and (pm == 0).all() and np.array_equal(I.unpack_bits_lsb(b, 96), clean.payload)
    b2, _, ok2, _ = oracle_mod.decode(fr, 4, clean.llr_f32, 32, I.CRC32_POLY, m)
    info = I.info_positions(fr)
    u = I.polar_transform(clean.codeword)
    assert np.array_equal(I.unpack_bits_lsb(b2, 96), u[:, info[:96]])
    # noisy frames: the systematic payload is x at the information positions of
    # the word the decoder returns, and errors are no more frequent than u-errors
    f = I.make_frames(fr, 32, I.CRC32_POLY, 2.0, 300, seed=3, systematic=True)
    b, _, ok, _ = oracle_mod.decode(fr, 8, f.llr_f32, 32, I.CRC32_POLY, m | oracle_mod.SYSTEMATIC)
    err = (I.unpack_bits_lsb(b, 96) != f.payload).any(axis=1)
    assert err.mean() < 0.5 and (ok[~err] == 1).all()


def _chase2_even(y, n_lrb=4):
    """Chase-II list of a single-parity-check code, written independently of
    the node rule: flip every subset of the n_lrb least reliable positions of
    the hard decision (ranked by |y|, then index), keep the even-weight words,
    and score each by the sum of |y| over the flipped positions."""
    y = np.asarray(y, np.float64)
    hd = (y < 0).astype(np.uint8)
    order = sorted(range(y.size), key=lambda i: (abs(float(y[i])), i))[:n_lrb]
    out = []
    for mask in range(1 << n_lrb):
        w = hd.copy()
        pen = 0.0
        for r in range(n_lrb):
            if (mask >> r) & 1:
                w[order[r]] ^= 1
                pen += abs(float(y[order[r]]))
        if int(w.sum()) % 2 == 0:
            out.append((pen, tuple(int(v) for v in w)))
    return sorted(out)


@pytest.mark.parametrize("N", [8, 16, 32])
def test_long_spc_nodes_equal_chase2(oracle_mod, N):
    # Dec-SPC-4+ (SPC nodes of any length, Sec. III-D): a code whose only
    # frozen bit is the first is one SPC node at the root; with L = 8 its final
    # list is every candidate, which must be the Chase-II list over the four
    # least reliable bits restricted to even weight
    fr = np.zeros(N, np.uint8)
    fr[0] = 1
    rng = np.random.default_rng(N)
    for _ in range(30):
        y = np.round(rng.normal(0, 3, N), 1).astype(np.float32)
        got = {w: p for p, w in _final_list(oracle_mod, fr, 8, y, oracle_mod.SPC_ANY)}
        want = {w: p for p, w in _chase2_even(y)}
        assert set(got) == set(want)                       # the same eight words
        for w in want:                                     # with the same metrics (float32 vs float64 sums)
            assert got[w] == pytest.approx(want[w], rel=1e-6, abs=1e-6)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_l2_spc_two_candidates_equal_all_eight(oracle_mod, dtype):
    """Sec. III-D: at L = 2 an SPC node needs only its first two candidates.
    Under the key (penalty, source, candidate) they are each source's two best
    (the others add least-reliable-bit terms at least as large), so the two
    survivors of all eight candidates are the same paths in the same slots."""
    rng = np.random.default_rng(212)
    with_spc = 0
    for mode in (oracle_mod.SPC4, oracle_mod.SPC_ANY):
        for N in (16, 32, 64, 128, 256):
            for _ in range(3):
                K = int(rng.integers(N // 4, N - 2))
                crc = 8 if K > 12 else 0
                fr = I.ga_frozen_mask(N, K, float(rng.uniform(0, 3)), max(K - crc, 1) / N)
                f = I.make_frames(fr, crc, I.CRC8_POLY, float(rng.uniform(-1, 2.5)), 60,
                                  seed=int(rng.integers(1 << 30)))
                llr = f.llr_i8 if dtype == "i8" else f.llr_f32
                if dtype == "i8":
                    llr[:10] = rng.integers(-3, 4, (10, N))          # many ties
                two = oracle_mod.decode(fr, 2, llr, crc, I.CRC8_POLY, mode)
                eight = oracle_mod.decode(fr, 2, llr, crc, I.CRC8_POLY, mode | oracle_mod.SPC_ALL_CANDIDATES)
                for a, b in zip(two, eight):
                    assert np.array_equal(a, b), (mode, N, K)
                with_spc += any(op[0] == oracle_mod.LEAF_SPC for op in oracle_mod.schedule(fr, mode))
    assert with_spc >= 15
    # an unknown flag bit is still refused
    with pytest.raises(Exception):
        oracle_mod.decode(I.ga_frozen_mask(16, 8, 2.0), 2, np.zeros((1, 16), np.float32), 0, 0, 0x400)
