"""CPU oracle for polar list-CRC decoding -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper over ``polar_oracle.c``: a plain bit-by-bit LLR SC-list
decoder and a plain version of the paper's fast list decoder (Rate-0,
Rate-1, repetition and SPC list nodes), both with full path copies. Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
use it; the product decoder never does.

Modes: ``BITWISE`` (SC-list, length-one leaves), ``SPC4`` (the paper's
"Dec-SPC-4"), ``SPC_ANY`` ("Dec-SPC-4+"); any of them | ``SYSTEMATIC`` for a
systematic code. ``SPC_ANY``'s long SPC nodes are not exhaustive; the tests
pin them against an independent Chase-II enumeration instead of brute-force ML.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

SPC4, SPC_ANY, BITWISE = 0, 1, 2
SYSTEMATIC = 0x100   # or-ed into a mode: payload and CRC read from x, not u = x G_N
SPC_ALL_CANDIDATES = 0x200   # tests only: all eight SPC candidates even at L = 2
F32, I8 = 0, 1
OP_F, OP_G, OP_COMBINE = 0, 1, 2
LEAF_RATE0, LEAF_RATE1, LEAF_REP, LEAF_SPC = 11, 12, 13, 14

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polar_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
        lib.oracle_decode.argtypes = [i, i, vp, i, i, i, i, u64, vp, i, vp, vp, vp, vp, i]
        lib.oracle_decode.restype = i
        lib.oracle_decode_list.argtypes = [i, i, vp, i, i, i, vp, vp, vp, vp]
        lib.oracle_decode_list.restype = i
        lib.oracle_schedule.argtypes = [i, vp, i, vp, i]
        lib.oracle_schedule.restype = i
        lib.oracle_crc.argtypes = [vp, i, u64, i, u64]
        lib.oracle_crc.restype = u64
        lib.oracle_polar_transform.argtypes = [vp, i]
        lib.oracle_polar_transform.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _llr_array(llr, dtype):
    if dtype == I8:
        return np.ascontiguousarray(llr, dtype=np.int8)
    return np.ascontiguousarray(llr, dtype=np.float32)


def decode(frozen, L, llr, crc_len=0, crc_poly=0, mode=SPC4, n_threads=1):
    """Decode frames. ``llr`` is float32 or int8 [F, N]; the dtype picks the mode.

    Returns (payload_bits_packed [F, ceil(k/8)], penalty [F], crc_ok [F], slot [F]).
    """
    lib = _load()
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    N = frozen.size
    K = int((frozen == 0).sum())
    llr = np.asarray(llr)
    dtype = I8 if llr.dtype == np.int8 else F32
    llr = _llr_array(llr, dtype).reshape(-1, N)
    F = llr.shape[0]
    k = K - crc_len
    bits = np.zeros((F, (k + 7) // 8), dtype=np.uint8)
    pm = np.zeros(F, dtype=np.float32)
    ok = np.zeros(F, dtype=np.uint8)
    slot = np.zeros(F, dtype=np.int32)
    rc = lib.oracle_decode(N, K, _ptr(frozen), L, dtype, mode, crc_len, crc_poly, _ptr(llr), F,
                           _ptr(bits), _ptr(pm), _ptr(ok), _ptr(slot), n_threads)
    if rc != 0:
        raise ValueError("oracle_decode rejected its arguments")
    return bits, pm, ok, slot


def adaptive_decode(frozen, L_max, llr, crc_len, crc_poly, mode=SPC4, n_threads=1):
    """Adaptive decoding of Sec. V: Fast-SSC (the list decoder with one path)
    on every frame, then the list decoder with ``L_max`` on the frames whose
    CRC failed. Returns decode()'s four arrays plus the re-decoded count."""
    llr = np.asarray(llr)
    N = np.asarray(frozen).size
    flat = llr.reshape(-1, N)
    bits, pm, ok, slot = decode(frozen, 1, flat, crc_len, crc_poly, mode, n_threads)
    bad = np.flatnonzero(ok == 0)
    if bad.size:
        b2, p2, o2, s2 = decode(frozen, L_max, flat[bad], crc_len, crc_poly, mode, n_threads)
        bits[bad], pm[bad], ok[bad], slot[bad] = b2, p2, o2, s2
    return bits, pm, ok, slot, int(bad.size)


def decode_list(frozen, L, llr_frame, mode=SPC4):
    """Final list of one frame: (codewords uint8 [n, N], penalties float32 [n])."""
    lib = _load()
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    N = frozen.size
    K = int((frozen == 0).sum())
    llr = np.asarray(llr_frame)
    dtype = I8 if llr.dtype == np.int8 else F32
    llr = _llr_array(llr, dtype).reshape(N)
    words = np.zeros((L, N), dtype=np.uint8)
    pens = np.zeros(L, dtype=np.float32)
    nf = ctypes.c_int(0)
    rc = lib.oracle_decode_list(N, K, _ptr(frozen), L, dtype, mode, _ptr(llr), _ptr(words),
                                _ptr(pens), ctypes.byref(nf))
    if rc != 0:
        raise ValueError("oracle_decode_list rejected its arguments")
    return words[: nf.value], pens[: nf.value]


def schedule(frozen, mode=SPC4):
    """Unrolled operation list [(kind, N_v, first u index), ...]."""
    lib = _load()
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    cap = 4 * frozen.size + 8
    ops = np.zeros(3 * cap, dtype=np.int32)
    n = lib.oracle_schedule(frozen.size, _ptr(frozen), mode, _ptr(ops), cap)
    if n < 0:
        raise ValueError("oracle_schedule failed")
    return [tuple(int(v) for v in ops[3 * i: 3 * i + 3]) for i in range(n)]


def crc(bits, crc_len, poly, init=0) -> int:
    lib = _load()
    b = np.ascontiguousarray(bits, dtype=np.uint8)
    return int(lib.oracle_crc(_ptr(b), b.size, poly, crc_len, init))


def polar_transform(v) -> np.ndarray:
    lib = _load()
    b = np.array(v, dtype=np.uint8, copy=True)
    lib.oracle_polar_transform(_ptr(b), b.size)
    return b
