"""Pins for the seeded input generator (CPU only).

The generator is shared by the CUDA decoder's tests and the oracle's, so it
is pinned against things outside itself: CRC catalogue check values and
zlib, the Kronecker-product definition of G_N, the (8,4) example of Fig. 1,
scipy quadrature and the large-mean asymptote of phi, and the AWGN moments.
"""
import math
import zlib

import numpy as np
import pytest

from paper_1505_01466_gb300 import inputs as I

CHECK = np.unpackbits(np.frombuffer(b"123456789", dtype=np.uint8))  # MSB-first per byte


def test_crc_catalogue_values():
    # CRC-8/SMBUS (poly 0x07, init 0, no reflection, no xor-out): check 0xF4.
    assert int("".join(map(str, I.crc_bits(CHECK, 8, 0x07))), 2) == 0xF4
    # CRC-32/MPEG-2 (poly 0x04C11DB7, init 0xFFFFFFFF, no reflection): 0x0376E6E7.
    v = int("".join(map(str, I.crc_bits(CHECK, 32, I.CRC32_POLY, init=0xFFFFFFFF))), 2)
    assert v == 0x0376E6E7
    # CRC-32/POSIX has init 0 and xor-out 0xFFFFFFFF with check 0x765E7680, so
    # the variant used here (init 0, no xor-out) must give 0x765E7680 ^ ~0.
    v = int("".join(map(str, I.crc_bits(CHECK, 32, I.CRC32_POLY))), 2)
    assert v == 0x765E7680 ^ 0xFFFFFFFF


def _reflect(v, w):
    return int(format(v, f"0{w}b")[::-1], 2)


def test_crc32_matches_zlib_after_reflection():
    rng = np.random.default_rng(5)
    for n in (1, 7, 64, 300):
        data = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        bits_lsb_first = np.unpackbits(np.frombuffer(data, np.uint8), bitorder="little")
        reg = int("".join(map(str, I.crc_bits(bits_lsb_first, 32, I.CRC32_POLY, 0xFFFFFFFF))), 2)
        assert _reflect(reg, 32) ^ 0xFFFFFFFF == zlib.crc32(data)


def test_crc_appended_word_has_zero_remainder_and_is_linear():
    rng = np.random.default_rng(1)
    d = rng.integers(0, 2, (20, 100), dtype=np.uint8)
    r = I.crc_bits(d, 32, I.CRC32_POLY)
    full = np.concatenate([d, r], axis=1)
    assert not I.crc_bits(full, 32, I.CRC32_POLY).any()
    a, b = d[:10], d[10:]
    assert np.array_equal(I.crc_bits(a ^ b, 32, I.CRC32_POLY),
                          I.crc_bits(a, 32, I.CRC32_POLY) ^ I.crc_bits(b, 32, I.CRC32_POLY))


@pytest.mark.parametrize("N", [2, 8, 32, 256])
def test_polar_transform_is_kronecker_power(N):
    F = np.array([[1, 0], [1, 1]], dtype=np.int64)
    G = np.array([[1]], dtype=np.int64)
    while G.shape[0] < N:
        G = np.kron(G, F)
    rng = np.random.default_rng(N)
    u = rng.integers(0, 2, (16, N), dtype=np.uint8)
    assert np.array_equal(I.polar_transform(u), (u.astype(np.int64) @ G) % 2)
    assert np.array_equal(I.polar_transform(I.polar_transform(u)), u)   # G_N G_N = I


def test_ga_information_set_of_fig1():
    mask = I.ga_frozen_mask(8, 4, 2.0)
    assert list(I.info_positions(mask)) == [3, 5, 6, 7]


def test_phi_against_scipy_quadrature_and_asymptote():
    integrate = pytest.importorskip("scipy.integrate")
    for m in (0.05, 0.5, 2.0, 10.0, 40.0):
        s = math.sqrt(2 * m)
        f = lambda u: (1.0 - math.tanh(u / 2)) * math.exp(-(u - m) ** 2 / (4 * m)) / math.sqrt(4 * math.pi * m)
        ref, _ = integrate.quad(f, m - 30 * s, m + 30 * s, points=[0.0], limit=400, epsabs=0, epsrel=1e-12)
        lp, psi = I._log_phi_and_psi(m)
        assert math.exp(lp) == pytest.approx(ref, rel=1e-6)
        assert psi == pytest.approx(1.0 - ref, rel=1e-6, abs=1e-12)
    # large-mean asymptote phi(m) ~ sqrt(pi/m) exp(-m/4) (1 - 10/(7m)) + O(m^-2)
    for m in (200.0, 1000.0, 20000.0):
        lp, _ = I._log_phi_and_psi(m)
        asym = 0.5 * math.log(math.pi / m) - m / 4 + math.log(1 - 10 / (7 * m))
        assert abs(lp - asym) < 5.0 / m


def test_ga_means_monotone_and_doubling():
    means = I.ga_leaf_means(64, 3.0, 0.5)
    # a right (G) child doubles its parent's mean, a left (F) child is below it
    assert (means[1::2] >= means[0::2]).all()
    sig = I.sigma_for(3.0, 0.5)
    assert means[-1] == pytest.approx(64 * 2 / sig ** 2)


def test_awgn_llr_moments_and_quantisation():
    fr = I.ga_frozen_mask(256, 128, 2.0)
    f = I.make_frames(fr, 0, 0, 2.0, 400, seed=3)
    sig = f.sigma
    s = 1.0 - 2.0 * f.codeword.astype(np.float64)
    z = f.llr_f32.astype(np.float64) * s          # sign-corrected LLR ~ N(2/s^2, 4/s^2)
    assert z.mean() == pytest.approx(2 / sig ** 2, rel=0.02)
    assert z.var() == pytest.approx(4 / sig ** 2, rel=0.03)
    q = I.quantize_i8(np.array([0.125, 0.375, -0.125, -0.375, 100.0, -100.0, 1.0]))
    assert list(q) == [0, 2, 0, -2, 127, -127, 4]   # rint: half to even


def test_noiseless_frames_and_payload_placement():
    fr = I.ga_frozen_mask(64, 40, 3.0)
    f = I.make_frames(fr, 8, I.CRC8_POLY, 3.0, 10, seed=9, noiseless=True)
    u = I.polar_transform(f.codeword)
    info = I.info_positions(fr)
    assert not u[:, fr == 1].any()
    assert np.array_equal(u[:, info[:32]], f.payload)
    assert not I.crc_bits(u[:, info], 8, I.CRC8_POLY).any()
    assert np.array_equal(f.llr_f32 < 0, f.codeword == 1)


def test_pack_roundtrip():
    rng = np.random.default_rng(0)
    b = rng.integers(0, 2, (3, 13), dtype=np.uint8)
    p = I.pack_bits_lsb(b)
    assert p.shape == (3, 2)
    assert p[0, 0] == sum(int(b[0, i]) << i for i in range(8))
    assert np.array_equal(I.unpack_bits_lsb(p, 13), b)


def test_batch_zipf_mix_counts():
    classes = I.batch_classes()
    assert len(classes) == 125
    counts = I.zipf_class_counts(1 << 20, 125, seed=1)
    assert counts.sum() == 1 << 20 and (counts > 0).all()
    assert counts.max() / counts.min() > 100          # uneven (Zipf s = 1.2)
    fc = I.frame_order(counts, seed=1)
    assert np.array_equal(np.bincount(fc, minlength=125), counts)


def test_chunked_frames_are_the_concatenated_chunks():
    fr = I.ga_frozen_mask(128, 70, 2.0, 62 / 128)
    full = I.make_frames_chunked(fr, 8, I.CRC8_POLY, 2.0, 50, seed=3, chunk=16, threads=3)
    one = I.make_frames_chunked(fr, 8, I.CRC8_POLY, 2.0, 50, seed=3, chunk=16, threads=1)
    assert np.array_equal(full.llr_f32, one.llr_f32) and full.payload.shape == (50, 62)
    c2 = I.make_frames(fr, 8, I.CRC8_POLY, 2.0, 16, seed=(3 << 20) + 2)
    assert np.array_equal(full.llr_i8[32:48], c2.llr_i8) and np.array_equal(full.payload[32:48], c2.payload)


def test_systematic_encoder_places_data_in_the_codeword():
    for N, K, db in ((64, 40, 3.0), (1024, 860, 4.0), (2048, 1723, 4.0)):
        fr = I.ga_frozen_mask(N, K, db)
        f = I.make_frames(fr, 32, I.CRC32_POLY, db, 20, seed=N, noiseless=True, systematic=True)
        info = I.info_positions(fr)
        x = f.codeword
        assert np.array_equal(x[:, info[: K - 32]], f.payload)          # payload in x itself
        assert not I.crc_bits(x[:, info], 32, I.CRC32_POLY).any()        # CRC in x too
        assert not I.polar_transform(x)[:, fr == 1].any()                # still a codeword of the code
        # the non-systematic encoding of the same data differs (but is also a codeword)
        g = I.make_frames(fr, 32, I.CRC32_POLY, db, 20, seed=N, noiseless=True)
        assert np.array_equal(g.payload, f.payload) and not np.array_equal(g.codeword, f.codeword)


def test_torch_frames_follow_the_same_construction():
    torch = pytest.importorskip("torch")
    fr = I.ga_frozen_mask(128, 72, 2.0, 64 / 128)
    info = I.info_positions(fr)
    pay, f32, i8 = I.make_frames_torch(fr, 8, I.CRC8_POLY, 2.0, 600, seed=9, device="cpu", chunk=256)
    pay, f32, i8 = pay.numpy(), f32.numpy(), i8.numpy()
    # the CRC matrix is the CRC of unit vectors, and linearity gives every CRC
    C = I.crc_generator_matrix(64, 8, I.CRC8_POLY)
    assert np.array_equal((pay.astype(np.int64) @ C) % 2, I.crc_bits(pay, 8, I.CRC8_POLY))
    # at a very high Eb/N0 the hard decisions are the codeword: its u carries
    # the payload and the CRC at the information positions and zeros elsewhere
    pay2, f2, _ = I.make_frames_torch(fr, 8, I.CRC8_POLY, 60.0, 50, seed=4, device="cpu")
    x = (f2.numpy() < 0).astype(np.uint8)
    u = I.polar_transform(x)
    assert not u[:, fr == 1].any()
    assert np.array_equal(u[:, info[:64]], pay2.numpy())
    assert np.array_equal(u[:, info[64:]], I.crc_bits(pay2.numpy(), 8, I.CRC8_POLY))
    # LLR = 2 y / sigma^2 with y = (1 - 2x) + sigma n: mean 2/sigma^2 * (1 - 2x), variance 4/sigma^2
    sig = I.sigma_for(2.0, 64 / 128)
    z = f32 * (sig * sig / 2.0)
    # recover the codeword from the payload to centre the noise
    u = np.zeros((600, 128), np.uint8)
    u[:, info[:64]] = pay
    u[:, info[64:]] = I.crc_bits(pay, 8, I.CRC8_POLY)
    xs = I.polar_transform(u)
    noise = (z - (1.0 - 2.0 * xs)) / sig
    assert abs(noise.mean()) < 0.01 and abs(noise.std() - 1.0) < 0.01
    # int8: rint(4 LLR) clamped to +-127
    want = np.clip(np.rint(f32.astype(np.float64) * 4.0), -127, 127)
    assert np.abs(i8.astype(np.float64) - want).max() <= 1.0
    assert (i8 == want).mean() > 0.999
    # a seed fixes the stream
    pay3, f3, _ = I.make_frames_torch(fr, 8, I.CRC8_POLY, 2.0, 600, seed=9, device="cpu", chunk=256)
    assert np.array_equal(pay3.numpy(), pay) and np.array_equal(f3.numpy(), f32)
