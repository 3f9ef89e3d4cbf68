"""Seeded synthetic inputs for polar list-CRC decoding.

This module only *makes inputs*: a frozen set, random CRC-protected payloads,
their polar codewords, and BPSK-over-AWGN channel LLRs (float32, or saturated
int8). It holds none of the decoding arithmetic, and both the CUDA decoder and
the CPU oracle read what it produces.

Conventions (Sec. II-A, II-B and VI of "Fast List Decoders for Polar Codes"):

* N = 2**n, natural bit order, codeword x = u * G_N with G_N = F^{(x)n},
  F = [[1, 0], [1, 1]] (the encoding graph of Fig. 1). No bit reversal.
* K counts the information positions *including* the CRC; the payload has
  k = K - crc_len bits. Payload bits fill the first k information positions
  (ascending index), the CRC fills the last crc_len positions.
* CRC: normal (MSB-first) polynomial division, initial register 0, no
  reflection, no final xor, computed over the payload bits in order.
* BPSK maps bit 0 to +1 and bit 1 to -1, so a positive LLR favours 0
  (the threshold rule h of Eq. (4)).
* Eb/N0 to noise: sigma^2 = 1 / (2 * R * 10**(EbN0/10)) with R = k / N, the
  payload rate (Sec. VI keeps the overall rate when a CRC is added).
* The frozen set is not given by the paper. It is built here by Gaussian-
  approximation density evolution at a design Eb/N0: every channel LLR has
  mean m0 = 2 / sigma^2, a left (F) child gets phi^{-1}(1 - (1 - phi(m))^2),
  a right (G) child gets 2 m, and the information set is the K leaves with
  the largest means (ties go to the higher index). phi is evaluated by
  numerical quadrature in double precision, not by a fitted formula.
"""

from __future__ import annotations

import functools
import math
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "CRC8_POLY", "CRC32_POLY", "crc_bits", "polar_transform", "ga_leaf_means",
    "ga_frozen_mask", "info_positions", "sigma_for", "Frames", "make_frames",
    "quantize_i8", "pack_bits_lsb", "unpack_bits_lsb", "crc_generator_matrix", "make_frames_torch",
]

CRC8_POLY = 0x07
CRC32_POLY = 0x04C11DB7


# --------------------------------------------------------------------------
# CRC (MSB-first, init 0, no reflection, no final xor), vectorised over rows.
# --------------------------------------------------------------------------
def crc_bits(bits: np.ndarray, crc_len: int, poly: int, init: int = 0) -> np.ndarray:
    """CRC register of each row of ``bits`` (shape [..., k], values 0/1).

    Returns the crc_len CRC bits of every row, most significant first, as a
    uint8 array of shape [..., crc_len]. ``init`` presets the register (only
    the catalogue checks in the tests use a non-zero value).
    """
    bits = np.asarray(bits, dtype=np.uint8)
    if crc_len == 0:
        return np.zeros(bits.shape[:-1] + (0,), dtype=np.uint8)
    if crc_len > 63:
        raise ValueError("crc_len must be <= 63")
    lead = bits.shape[:-1]
    flat = bits.reshape(-1, bits.shape[-1])
    mask = (1 << crc_len) - 1
    reg = np.full(flat.shape[0], init & mask, dtype=np.uint64)
    top_shift = np.uint64(crc_len - 1)
    p = np.uint64(poly & mask)
    m = np.uint64(mask)
    one = np.uint64(1)
    for t in range(flat.shape[1]):
        fb = ((reg >> top_shift) & one) ^ flat[:, t].astype(np.uint64)
        reg = ((reg << one) & m) ^ (fb * p)
    out = np.empty((flat.shape[0], crc_len), dtype=np.uint8)
    for b in range(crc_len):
        out[:, b] = ((reg >> np.uint64(crc_len - 1 - b)) & one).astype(np.uint8)
    return out.reshape(lead + (crc_len,))


# --------------------------------------------------------------------------
# Polar transform x = u G_N (natural order). G_N is its own inverse.
# --------------------------------------------------------------------------
def polar_transform(u: np.ndarray) -> np.ndarray:
    """x = u * G_N over GF(2) for every row of u (shape [..., N])."""
    x = np.array(u, dtype=np.uint8, copy=True)
    N = x.shape[-1]
    if N & (N - 1):
        raise ValueError("N must be a power of two")
    lead = x.shape[:-1]
    h = 1
    while h < N:
        v = x.reshape(lead + (N // (2 * h), 2, h))
        v[..., 0, :] ^= v[..., 1, :]
        h *= 2
    return x


# --------------------------------------------------------------------------
# Gaussian-approximation density evolution.
# --------------------------------------------------------------------------
def _log_phi_and_psi(m: float) -> tuple[float, float]:
    """log(phi(m)) and psi(m) = 1 - phi(m) for one mean m > 0.

    phi(m) = E[1 - tanh(U/2)] = E[2 / (1 + exp(U))], U ~ Normal(m, 2m).
    The integral is a trapezoid sum on a uniform grid, taken in the log
    domain so that phi can be far below the double-precision floor of 1.
    """
    s = math.sqrt(2.0 * m)
    if m <= 100.0:
        lo, hi = m - 20.0 * s, m + 20.0 * s
        h = min(0.02, s / 100.0)
    else:
        # For m > 100 the mass of 2/(1+e^u) * N(u; m, 2m) sits near u = 0;
        # the Gaussian bulk near u = m contributes about exp(-3m/4) relative.
        lo, hi = -60.0, 60.0
        h = 0.02
    npts = int(math.ceil((hi - lo) / h)) + 1
    u = np.linspace(lo, hi, npts)
    step = (hi - lo) / (npts - 1)
    log_gauss = -((u - m) ** 2) / (4.0 * m) - 0.5 * math.log(4.0 * math.pi * m)
    log_f = math.log(2.0) - np.logaddexp(0.0, u) + log_gauss
    w = np.full(npts, step)
    w[0] = w[-1] = step / 2.0
    lw = log_f + np.log(w)
    mx = lw.max()
    log_phi = float(mx + math.log(np.exp(lw - mx).sum()))
    if m <= 100.0:
        psi = float((np.tanh(u / 2.0) * np.exp(log_gauss) * w).sum())
    else:
        psi = -math.expm1(log_phi)
    return log_phi, psi


@functools.lru_cache(maxsize=1)
def _phi_table():
    logm = np.linspace(math.log(1e-12), math.log(1e6), 2401)
    lp = np.empty_like(logm)
    ps = np.empty_like(logm)
    for i, lm in enumerate(logm):
        lp[i], ps[i] = _log_phi_and_psi(math.exp(lm))
    # psi is increasing and log(phi) decreasing in m; enforce strict
    # monotonicity against round-off at the flat ends before inversion.
    ps = np.maximum.accumulate(ps)
    lp = np.minimum.accumulate(lp)
    return logm, lp, np.log(np.maximum(ps, 1e-300))


def _f_child_mean(m: np.ndarray) -> np.ndarray:
    """Mean of the left (F) child: phi^{-1}(1 - (1 - phi(m))^2).

    In terms of psi = 1 - phi this reads psi(m_l) = psi(m)^2, which is well
    conditioned for small means; for large means the equivalent form
    log phi(m_l) = log phi(m) + log(2 - phi(m)) is used.
    """
    logm, lp, lps = _phi_table()
    lm = np.log(m)
    out = np.empty_like(m)
    lp_m = np.interp(lm, logm, lp)
    lps_m = np.interp(lm, logm, lps)
    phi_m = np.exp(lp_m)
    tgt_lps = 2.0 * lps_m                                     # log psi target
    tgt_lp = lp_m + np.log(2.0 - phi_m)                        # log phi target
    use_psi = tgt_lps < math.log(0.5)
    # invert psi (increasing): interp over (lps, logm)
    below = use_psi & (tgt_lps < lps[0])
    out_psi = np.exp(np.interp(tgt_lps, lps, logm))
    # below the table psi(m) ~ m/2, so m ~ 2 psi
    out_psi = np.where(below, 2.0 * np.exp(tgt_lps), out_psi)
    # invert log phi (decreasing): interp over reversed arrays
    out_phi = np.exp(np.interp(-tgt_lp, -lp, logm))
    out[:] = np.where(use_psi, out_psi, out_phi)
    return out


def sigma_for(ebn0_db: float, rate: float) -> float:
    """Noise standard deviation for BPSK at Eb/N0 (dB) and payload rate."""
    return math.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0)))


def ga_leaf_means(N: int, design_ebn0_db: float, rate: float) -> np.ndarray:
    """LLR means of the N synthetic channels u_0..u_{N-1} (natural order)."""
    if N < 1 or N & (N - 1):
        raise ValueError("N must be a power of two")
    sig = sigma_for(design_ebn0_db, rate)
    m = np.array([2.0 / (sig * sig)])
    while m.size < N:
        nxt = np.empty(2 * m.size)
        nxt[0::2] = _f_child_mean(m)
        nxt[1::2] = 2.0 * m
        m = nxt
    return m


def ga_frozen_mask(N: int, K: int, design_ebn0_db: float, rate: float | None = None) -> np.ndarray:
    """uint8[N] with 1 at frozen positions: the N-K least reliable channels.

    ``rate`` is the payload rate used for the design noise level (defaults to
    K/N, i.e. no CRC).
    """
    if not 0 <= K <= N:
        raise ValueError("need 0 <= K <= N")
    if rate is None:
        rate = K / N
    means = ga_leaf_means(N, design_ebn0_db, rate)
    # Sort by (mean, index) descending: ties go to the higher index.
    order = np.lexsort((np.arange(N), means))[::-1]
    mask = np.ones(N, dtype=np.uint8)
    mask[order[:K]] = 0
    return mask


def info_positions(frozen_mask: np.ndarray) -> np.ndarray:
    return np.flatnonzero(np.asarray(frozen_mask) == 0).astype(np.int64)


# --------------------------------------------------------------------------
# Frames: payload -> CRC -> u -> x -> BPSK + AWGN -> LLR.
# --------------------------------------------------------------------------
@dataclass
class Frames:
    payload: np.ndarray      # uint8 [F, k]
    codeword: np.ndarray     # uint8 [F, N]
    llr_f32: np.ndarray      # float32 [F, N]
    llr_i8: np.ndarray       # int8 [F, N]
    sigma: float


def quantize_i8(llr: np.ndarray, scale: float = 4.0) -> np.ndarray:
    """q = clamp(rint(scale * LLR), -127, 127), rint = round half to even."""
    q = np.rint(np.asarray(llr, dtype=np.float64) * scale)
    return np.clip(q, -127, 127).astype(np.int8)


def systematic_encode(v: np.ndarray, frozen_mask: np.ndarray) -> np.ndarray:
    """Systematic polar encoding: v holds the information bits at the
    information positions (zeros elsewhere); x = ((v G_N) with the frozen
    positions cleared) G_N. For information sets closed under the polar
    order (those of density evolution are) x equals v at every information
    position."""
    w = polar_transform(v)
    w[..., np.asarray(frozen_mask) == 1] = 0
    return polar_transform(w)


def make_frames(frozen_mask: np.ndarray, crc_len: int, crc_poly: int, ebn0_db: float,
                n_frames: int, seed: int, noiseless: bool = False, systematic: bool = False) -> Frames:
    """Random codewords of the polar-CRC code sent over BPSK-AWGN.

    Uses numpy's counter-based Philox generator keyed by ``seed``. With
    ``noiseless`` the channel output is exactly +-1 (LLR = +-2/sigma^2). With
    ``systematic`` the payload and CRC are placed in the codeword itself.
    """
    frozen_mask = np.asarray(frozen_mask, dtype=np.uint8)
    N = frozen_mask.size
    info = info_positions(frozen_mask)
    K = info.size
    k = K - crc_len
    if k < 0:
        raise ValueError("crc_len larger than K")
    rng = np.random.Generator(np.random.Philox(key=np.uint64(seed)))
    payload = rng.integers(0, 2, size=(n_frames, k), dtype=np.uint8)
    crc = crc_bits(payload, crc_len, crc_poly)
    u = np.zeros((n_frames, N), dtype=np.uint8)
    u[:, info[:k]] = payload
    u[:, info[k:]] = crc
    x = systematic_encode(u, frozen_mask) if systematic else polar_transform(u)
    rate = k / N if k > 0 else K / N if K > 0 else 1.0 / N
    sig = sigma_for(ebn0_db, rate)
    y = 1.0 - 2.0 * x.astype(np.float64)
    if not noiseless:
        y = y + sig * rng.standard_normal((n_frames, N))
    llr = 2.0 * y / (sig * sig)
    return Frames(payload=payload, codeword=x, llr_f32=llr.astype(np.float32),
                  llr_i8=quantize_i8(llr), sigma=sig)


def make_frames_chunked(frozen_mask: np.ndarray, crc_len: int, crc_poly: int, ebn0_db: float,
                        n_frames: int, seed: int, chunk: int = 8192, threads: int | None = None,
                        systematic: bool = False) -> Frames:
    """make_frames over chunks of ``chunk`` frames generated on host threads.

    Chunk c is ``make_frames(..., chunk, seed=(seed << 20) + c)``; the result is
    their concatenation, so it does not depend on the thread count.
    """
    from concurrent.futures import ThreadPoolExecutor
    if n_frames == 0:
        return make_frames(frozen_mask, crc_len, crc_poly, ebn0_db, 0, seed)
    sizes = [min(chunk, n_frames - s) for s in range(0, n_frames, chunk)]
    threads = threads or min(len(sizes), os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda c: make_frames(frozen_mask, crc_len, crc_poly, ebn0_db, sizes[c],
                                                  seed=(seed << 20) + c, systematic=systematic),
                            range(len(sizes))))
    return Frames(payload=np.concatenate([p.payload for p in parts]),
                  codeword=np.concatenate([p.codeword for p in parts]),
                  llr_f32=np.concatenate([p.llr_f32 for p in parts]),
                  llr_i8=np.concatenate([p.llr_i8 for p in parts]), sigma=parts[0].sigma)


def crc_generator_matrix(k: int, crc_len: int, crc_poly: int) -> np.ndarray:
    """CRC bits of each unit payload vector e_t, uint8 [k, crc_len]. With a
    zero initial register and no final xor the CRC is linear over GF(2), so
    the CRC of a payload p is p C mod 2."""
    return crc_bits(np.eye(k, dtype=np.uint8), crc_len, crc_poly)


def make_frames_torch(frozen_mask: np.ndarray, crc_len: int, crc_poly: int, ebn0_db: float,
                      n_frames: int, seed: int, device, chunk: int = 1 << 17):
    """The frames of make_frames, generated with torch on ``device`` for
    Monte-Carlo sweeps of millions of frames: random payload bits, the CRC
    as p C mod 2 (crc_generator_matrix, exact in float64), u at the
    information positions, x = u G_N by butterflies, BPSK, float32 Gaussian
    noise from torch's generator seeded with ``seed``, LLR = 2 y / sigma^2,
    and the int8 quantisation of quantize_i8 applied to the float32 LLRs.

    Returns (payload uint8 [F, k], llr_f32 float32 [F, N], llr_i8 int8 [F, N]),
    all on ``device``. The streams differ from make_frames' (another
    generator), the construction is the same.
    """
    import torch
    frozen_mask = np.asarray(frozen_mask, dtype=np.uint8)
    N = frozen_mask.size
    info = info_positions(frozen_mask)
    K = info.size
    k = K - crc_len
    if k < 0:
        raise ValueError("crc_len larger than K")
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    C = torch.from_numpy(crc_generator_matrix(k, crc_len, crc_poly).astype(np.float64)).to(dev)
    info_pay = torch.from_numpy(info[:k]).to(dev)
    info_crc = torch.from_numpy(info[k:]).to(dev)
    rate = k / N if k > 0 else K / N if K > 0 else 1.0 / N
    sig = sigma_for(ebn0_db, rate)
    payload = torch.empty((n_frames, k), dtype=torch.uint8, device=dev)
    llr_f32 = torch.empty((n_frames, N), dtype=torch.float32, device=dev)
    llr_i8 = torch.empty((n_frames, N), dtype=torch.int8, device=dev)
    for s in range(0, n_frames, chunk):
        n = min(chunk, n_frames - s)
        p = torch.randint(0, 2, (n, k), generator=gen, device=dev, dtype=torch.uint8)
        u = torch.zeros((n, N), dtype=torch.uint8, device=dev)
        u[:, info_pay] = p
        if crc_len:
            u[:, info_crc] = torch.remainder(p.to(torch.float64) @ C, 2.0).to(torch.uint8)
        h = 1
        while h < N:
            v = u.view(n, N // (2 * h), 2, h)
            v[:, :, 0, :] ^= v[:, :, 1, :]
            h *= 2
        y = 1.0 - 2.0 * u.to(torch.float32)
        y += sig * torch.randn((n, N), generator=gen, device=dev, dtype=torch.float32)
        llr = y * (2.0 / (sig * sig))
        payload[s: s + n] = p
        llr_f32[s: s + n] = llr
        llr_i8[s: s + n] = torch.clamp(torch.round(llr * 4.0), -127, 127).to(torch.int8)
    return payload, llr_f32, llr_i8


# --------------------------------------------------------------------------
# Bit packing used by the output format (LSB-first within each byte).
# --------------------------------------------------------------------------
def pack_bits_lsb(bits: np.ndarray) -> np.ndarray:
    return np.packbits(np.asarray(bits, dtype=np.uint8), axis=-1, bitorder="little")


def unpack_bits_lsb(packed: np.ndarray, nbits: int) -> np.ndarray:
    return np.unpackbits(np.asarray(packed, dtype=np.uint8), axis=-1, count=nbits,
                         bitorder="little")


# --------------------------------------------------------------------------
# Mixed-code workloads (batched and serving forms).
# --------------------------------------------------------------------------
BATCH_NS = (256, 512, 1024, 2048, 4096)
BATCH_RATES = (0.25, 0.5, 0.75, 0.84, 0.9)
BATCH_LS = (2, 4, 8, 16, 32)


def batch_classes(ns=BATCH_NS, rates=BATCH_RATES, ls=BATCH_LS):
    """(N, K, L) for every class; K = round(rate * N) counts the CRC."""
    return [(N, int(round(r * N)), L) for N in ns for r in rates for L in ls]


def zipf_class_counts(n_frames: int, n_classes: int, seed: int, s: float = 1.2) -> np.ndarray:
    """Frame count per class: Zipf(s) over class ranks, the ranks being a seeded
    permutation of the classes; counts sum to n_frames (largest remainders)."""
    rng = np.random.Generator(np.random.Philox(key=np.uint64(seed)))
    rank_of = rng.permutation(n_classes)            # class c has rank rank_of[c] (0 = most frequent)
    w = 1.0 / (rank_of + 1.0) ** s
    p = w / w.sum()
    raw = p * n_frames
    counts = np.floor(raw).astype(np.int64)
    rem = n_frames - int(counts.sum())
    order = np.argsort(-(raw - counts), kind="stable")
    counts[order[:rem]] += 1
    return counts


def frame_order(counts: np.ndarray, seed: int) -> np.ndarray:
    """Class index of every frame, shuffled in arrival order (seeded)."""
    rng = np.random.Generator(np.random.Philox(key=np.uint64(seed + 1)))
    fc = np.repeat(np.arange(counts.size, dtype=np.uint32), counts)
    rng.shuffle(fc)
    return fc
