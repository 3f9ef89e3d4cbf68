"""Synthetic mixed-code workloads for the batched and serving forms.

Builds, from the seeded generators in ``inputs``, the 125 code classes
(N in {256..4096} x rate in {0.25, 0.5, 0.75, 0.84, 0.9} x L in {2..32},
CRC-32 inside K, frozen sets by GA at 4 dB) with a pool of noisy frames per
class. Only input preparation lives here: the decoding runs in the library.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I


class ClassPool:
    def __init__(self, N, K, L, crc_len, frozen, llr_f32, llr_i8, ebn0):
        self.N, self.K, self.L, self.crc_len = N, K, L, crc_len
        self.k = K - crc_len
        self.frozen = frozen
        self.llr_f32 = llr_f32
        self.llr_i8 = llr_i8
        self.ebn0 = ebn0

    def rows(self, start: int, n: int, dtype: str) -> np.ndarray:
        pool = self.llr_i8 if dtype == "i8" else self.llr_f32
        idx = (start + np.arange(n)) % pool.shape[0]
        return pool[idx]


def class_pools(pool_frames: int = 256, seed: int = 11, design_db: float = 4.0, ebn0s=(4.0,),
                crc_len: int = 32, classes=None):
    """One ClassPool per (N, K, L) class; frozen sets are shared across L."""
    classes = classes or I.batch_classes()
    frozen_cache = {}
    rng = np.random.default_rng(seed)
    pools = []
    for ci, (N, K, L) in enumerate(classes):
        key = (N, K)
        if key not in frozen_cache:
            frozen_cache[key] = I.ga_frozen_mask(N, K, design_db, (K - crc_len) / N)
        fr = frozen_cache[key]
        eb = float(ebn0s[int(rng.integers(len(ebn0s)))])
        f = I.make_frames(fr, crc_len, I.CRC32_POLY, eb, pool_frames, seed=seed * 1000 + ci)
        pools.append(ClassPool(N, K, L, crc_len, fr, f.llr_f32, f.llr_i8, eb))
    return pools
