"""Thin ctypes binding of ``libpolar_gb300.so`` (C ABI in include/polar.h).

Argument marshalling only: every step of the decode runs in the CUDA
kernels behind the C ABI. PyTorch supplies device memory and streams. There
is no CPU fallback -- if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpolar_gb300.so")

POLAR_OK, POLAR_EINVAL, POLAR_ENOMEM, POLAR_ECUDA = 0, -1, -2, -3
POLAR_EUNSUPPORTED, POLAR_ETIMEDOUT, POLAR_EBUSY = -4, -5, -6
LLR_F32, LLR_I8 = 0, 1
SPC_MAX_4, SPC_ANY, NO_SPECIAL_NODES, HOST_ONLY, SYSTEMATIC = 0, 1, 2, 0x100, 0x200
INJECT_ALLOC_FAIL, INJECT_POISON = 1, 2

# Every symbol include/polar.h declares.
EXPORTED = [
    "polar_code_create", "polar_code_destroy", "polar_list_decode", "polar_strerror", "polar_sync",
    "polar_code_get_info", "polar_code_schedule", "polar_code_op_count", "polar_code_set_launch",
    "polar_code_set_recompute", "polar_code_set_smem_budget", "polar_code_set_packing",
    "polar_code_autotune", "polar_list_decode_noalloc", "polar_noalloc_scratch_bytes",
    "polar_batch_plan", "polar_batch_destroy", "polar_batch_layout", "polar_batch_run", "polar_batch_set_launch",
    "polar_batch_autotune", "polar_batch_capture", "polar_batch_replay", "polar_batch_get_info",
    "polar_server_create", "polar_server_destroy", "polar_server_submit", "polar_server_poll", "polar_server_wait",
    "polar_server_pause", "polar_server_stats", "polar_server_latency", "polar_adaptive_decode", "polar_list_decode_host",
    "polar_debug_inject",
]


class PolarError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_lib().polar_strerror(status).decode()} ({status})")


class CodeInfo(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_uint32), ("K", ctypes.c_uint32), ("k", ctypes.c_uint32), ("L", ctypes.c_uint32),
        ("crc_len", ctypes.c_uint32), ("n_ops", ctypes.c_uint32), ("n_leaves", ctypes.c_uint32),
        ("n_rate0", ctypes.c_uint32), ("n_rate1", ctypes.c_uint32), ("n_rep", ctypes.c_uint32),
        ("n_spc", ctypes.c_uint32), ("warps_per_frame", ctypes.c_uint32 * 2),
        ("frames_per_cta", ctypes.c_uint32 * 2), ("smem_per_frame", ctypes.c_uint32 * 2),
        ("scratch_per_frame", ctypes.c_uint64 * 2), ("spill_mask", ctypes.c_uint32 * 2),
        ("recomputed_stages", ctypes.c_uint32 * 2), ("max_recompute_depth", ctypes.c_uint32),
        ("packed", ctypes.c_uint32 * 2),
    ]


def adaptive_decode(fast, list_code, llr, stream=None):
    """Sec. V adaptive decoding: ``fast`` (L = 1) first, CRC failures again with
    ``list_code``. Returns (bits, penalty, crc_ok, slot, n_relisted tensor)."""
    import torch
    dt = LLR_I8 if llr.dtype == torch.int8 else LLR_F32
    F = llr.numel() // fast.N
    dev = llr.device
    bits = torch.empty((F, (fast.k + 7) // 8), dtype=torch.uint8, device=dev)
    pm = torch.empty(F, dtype=torch.float32, device=dev)
    ok = torch.empty(F, dtype=torch.uint8, device=dev)
    slot = torch.empty(F, dtype=torch.int32, device=dev)
    nrel = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(_lib().polar_adaptive_decode(fast.handle, list_code.handle, ctypes.c_void_p(llr.data_ptr()), dt, F,
                                        ctypes.c_void_p(bits.data_ptr()), ctypes.c_void_p(pm.data_ptr()),
                                        ctypes.c_void_p(ok.data_ptr()), ctypes.c_void_p(slot.data_ptr()),
                                        ctypes.c_void_p(nrel.data_ptr()), _stream_handle(stream)),
           "polar_adaptive_decode")
    return bits, pm, ok, slot, nrel


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("n_frames", ctypes.c_uint32), ("n_codes", ctypes.c_uint32), ("warps_per_frame", ctypes.c_uint32),
        ("frames_per_cta", ctypes.c_uint32), ("smem_per_frame", ctypes.c_uint32), ("grid", ctypes.c_uint32),
        ("scratch_bytes", ctypes.c_uint64), ("llr_bytes", ctypes.c_uint64), ("bits_bytes", ctypes.c_uint64),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("completed", ctypes.c_uint64), ("frames", ctypes.c_uint64), ("info_bits", ctypes.c_uint64),
        ("pending", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("batches_in_flight", ctypes.c_uint64),
        ("batches", ctypes.c_uint64), ("max_batches_in_flight", ctypes.c_uint64),
        ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double),
        ("mean_us", ctypes.c_double), ("span_us", ctypes.c_double),
    ]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run paper_1505_01466_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        lib.polar_code_create.argtypes = [ctypes.POINTER(vp), u32, u32, vp, u32, u64, u32, u32]
        lib.polar_code_destroy.argtypes = [vp]
        lib.polar_list_decode.argtypes = [vp, vp, i32, u32, vp, vp, vp, vp, vp]
        lib.polar_strerror.argtypes = [i32]
        lib.polar_strerror.restype = ctypes.c_char_p
        lib.polar_sync.argtypes = [vp]
        lib.polar_code_get_info.argtypes = [vp, ctypes.POINTER(CodeInfo)]
        lib.polar_code_schedule.argtypes = [vp, vp, u32, ctypes.POINTER(u32)]
        lib.polar_code_op_count.argtypes = [vp, ctypes.POINTER(u64)]
        lib.polar_code_set_launch.argtypes = [vp, i32, u32, u32, u32]
        lib.polar_code_set_recompute.argtypes = [vp, i32, u32]
        lib.polar_code_set_packing.argtypes = [vp, i32, i32]
        lib.polar_code_set_smem_budget.argtypes = [vp, i32, u32]
        lib.polar_code_autotune.argtypes = [vp, i32, vp, u32, vp, ctypes.POINTER(u32), ctypes.POINTER(u32),
                                             ctypes.POINTER(u32)]
        lib.polar_list_decode_noalloc.argtypes = [vp, vp, i32, u32, vp, vp, vp, vp, vp]
        lib.polar_noalloc_scratch_bytes.argtypes = []
        lib.polar_batch_plan.argtypes = [ctypes.POINTER(vp), vp, u32, vp, u32, i32, u32]
        lib.polar_batch_destroy.argtypes = [vp]
        lib.polar_batch_layout.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), vp, vp]
        lib.polar_batch_run.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.polar_batch_set_launch.argtypes = [vp, u32, u32, u32]
        lib.polar_batch_autotune.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(u32), ctypes.POINTER(u32),
                                             ctypes.POINTER(u32)]
        lib.polar_batch_capture.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.polar_batch_replay.argtypes = [vp, vp]
        lib.polar_batch_get_info.argtypes = [vp, ctypes.POINTER(BatchInfo)]
        lib.polar_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, u32, u32, u32, u32]
        lib.polar_server_destroy.argtypes = [vp]
        lib.polar_server_submit.argtypes = [vp, vp, vp, i32, u32, ctypes.POINTER(u64)]
        lib.polar_server_poll.argtypes = [vp, u64, vp, vp, vp, ctypes.POINTER(i32)]
        lib.polar_server_wait.argtypes = [vp, u64, u32]
        lib.polar_server_pause.argtypes = [vp, i32]
        lib.polar_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats), i32]
        lib.polar_server_latency.argtypes = [vp, u32, u32, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]
        lib.polar_adaptive_decode.argtypes = [vp, vp, vp, i32, u32, vp, vp, vp, vp, vp, vp]
        lib.polar_list_decode_host.argtypes = [vp, vp, i32, u32, vp, vp, vp, vp, vp]
        lib.polar_debug_inject.argtypes = [i32, ctypes.c_int64]
        for name in EXPORTED:
            if name != "polar_strerror":
                getattr(lib, name).restype = i32
        lib.polar_noalloc_scratch_bytes.restype = ctypes.c_size_t
        _LIB = lib
    return _LIB


def load_library():
    """Load the C-ABI library (raises if it is not built)."""
    return _lib()


def sync(stream=None):
    """polar_sync: wait for ``stream`` (default: torch's current stream) and
    raise PolarError if asynchronous work on the device failed."""
    _check(_lib().polar_sync(_stream_handle(stream)), "polar_sync")


def debug_inject(what: int, value: int):
    """polar_debug_inject: host-side fault injection for tests."""
    _check(_lib().polar_debug_inject(what, value), "polar_debug_inject")


def _check(status: int, what: str):
    if status != POLAR_OK:
        raise PolarError(status, what)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class PolarCode:
    """A polar-CRC code prepared for list decoding on the GPU.

    frozen_mask: N bytes, nonzero = frozen. crc_len / crc_poly: the outer
    CRC (MSB-first, register starts at 0). L: list size (power of two <= 32).
    mode: SPC_MAX_4 (default), SPC_ANY or NO_SPECIAL_NODES. systematic: the
    payload and CRC sit in the codeword x (read from x, not from u = x G_N).
    """

    def __init__(self, frozen_mask, crc_len: int = 0, crc_poly: int = 0, L: int = 8,
                 mode: int = SPC_MAX_4, host_only: bool = False, systematic: bool = False):
        mask = np.ascontiguousarray(np.asarray(frozen_mask).astype(np.uint8) != 0, dtype=np.uint8)
        self.N = int(mask.size)
        self.K = int((mask == 0).sum())
        self.crc_len = int(crc_len)
        self.k = self.K - self.crc_len
        self.L = int(L)
        self.frozen = mask
        flags = int(mode) | (HOST_ONLY if host_only else 0) | (SYSTEMATIC if systematic else 0)
        h = ctypes.c_void_p()
        st = _lib().polar_code_create(ctypes.byref(h), self.N, self.K, mask.ctypes.data_as(ctypes.c_void_p),
                                      self.crc_len, int(crc_poly), self.L, flags)
        _check(st, "polar_code_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib().polar_code_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        ci = CodeInfo()
        _check(_lib().polar_code_get_info(self._h, ctypes.byref(ci)), "polar_code_get_info")
        out = {}
        for name, _ in CodeInfo._fields_:
            v = getattr(ci, name)
            out[name] = list(v) if hasattr(v, "__len__") else int(v)
        return out

    def schedule(self):
        n = ctypes.c_uint32(0)
        _lib().polar_code_schedule(self._h, None, 0, ctypes.byref(n))
        buf = np.zeros(3 * max(n.value, 1), dtype=np.int32)
        _check(_lib().polar_code_schedule(self._h, buf.ctypes.data_as(ctypes.c_void_p), n.value,
                                          ctypes.byref(n)), "polar_code_schedule")
        return [tuple(int(v) for v in buf[3 * i: 3 * i + 3]) for i in range(n.value)]

    def op_count(self) -> int:
        v = ctypes.c_uint64(0)
        _check(_lib().polar_code_op_count(self._h, ctypes.byref(v)), "polar_code_op_count")
        return int(v.value)

    def set_launch(self, dtype: int, warps_per_frame: int, smem_budget: int = 0, cta_threads: int = 0):
        _check(_lib().polar_code_set_launch(self._h, dtype, warps_per_frame, smem_budget, cta_threads),
               "polar_code_set_launch")

    def set_smem_budget(self, dtype: int, smem_per_warp: int):
        """Shared memory of the L = 1 kernel (per warp of 32 frames) or of a wide code (per CTA)."""
        _check(_lib().polar_code_set_smem_budget(self._h, dtype, smem_per_warp), "polar_code_set_smem_budget")

    def set_packing(self, dtype: int, on: bool):
        """L <= 16: register subtrees of 32 / L frames in one warp (lockstep rounds)."""
        _check(_lib().polar_code_set_packing(self._h, dtype, 1 if on else 0), "polar_code_set_packing")

    def set_recompute(self, dtype: int, depth: int):
        """Evaluate the top ``depth`` alpha stages from the channel instead of storing them."""
        _check(_lib().polar_code_set_recompute(self._h, dtype, depth), "polar_code_set_recompute")

    def autotune(self, llr, stream=None):
        """Time the launch shapes on ``llr`` ([F, N] CUDA tensor) and keep the fastest."""
        import torch
        dt = LLR_I8 if llr.dtype == torch.int8 else LLR_F32
        w, b, t = ctypes.c_uint32(0), ctypes.c_uint32(0), ctypes.c_uint32(0)
        _check(_lib().polar_code_autotune(self._h, dt, ctypes.c_void_p(llr.data_ptr()), llr.numel() // self.N,
                                          _stream_handle(stream), ctypes.byref(w), ctypes.byref(b), ctypes.byref(t)),
               "polar_code_autotune")
        return int(w.value), int(b.value), int(t.value)

    def decode_into(self, llr, bits, pm, ok=None, slot=None, stream=None):
        """Enqueue a decode of ``llr`` ([F, N] float32 or int8 CUDA tensor)."""
        import torch
        if llr.dtype == torch.float32:
            dt = LLR_F32
        elif llr.dtype == torch.int8:
            dt = LLR_I8
        else:
            raise TypeError("llr must be float32 or int8")
        if not llr.is_cuda or not llr.is_contiguous() or llr.shape[-1] != self.N:
            raise ValueError("llr must be a contiguous CUDA tensor [F, N]")
        F = llr.numel() // self.N
        st = _lib().polar_list_decode(
            self._h, ctypes.c_void_p(llr.data_ptr()), dt, F,
            ctypes.c_void_p(bits.data_ptr()), ctypes.c_void_p(pm.data_ptr()),
            ctypes.c_void_p(ok.data_ptr() if ok is not None else 0),
            ctypes.c_void_p(slot.data_ptr() if slot is not None else 0), _stream_handle(stream))
        _check(st, "polar_list_decode")

    def decode_host(self, llr, bits, pm, ok=None, slot=None, stream=None):
        """polar_list_decode_host: ``llr`` and the outputs are CPU tensors (pinned
        for overlapped copies); blocks until the outputs are written."""
        import torch
        dt = LLR_I8 if llr.dtype == torch.int8 else LLR_F32
        for t in (llr, bits, pm) + tuple(x for x in (ok, slot) if x is not None):
            if t.is_cuda or not t.is_contiguous():
                raise PolarError("decode_host takes contiguous host tensors")
        F = llr.numel() // self.N
        _check(_lib().polar_list_decode_host(self._h, ctypes.c_void_p(llr.data_ptr()), dt, F,
                                             ctypes.c_void_p(bits.data_ptr()), ctypes.c_void_p(pm.data_ptr()),
                                             ctypes.c_void_p(ok.data_ptr() if ok is not None else 0),
                                             ctypes.c_void_p(slot.data_ptr() if slot is not None else 0),
                                             _stream_handle(stream)), "polar_list_decode_host")

    def decode(self, llr, stream=None):
        """Decode; returns (payload bits [F, ceil(k/8)] uint8, penalty [F], crc_ok [F], slot [F])."""
        import torch
        F = llr.numel() // self.N
        dev = llr.device
        bits = torch.empty((F, (self.k + 7) // 8), dtype=torch.uint8, device=dev)
        pm = torch.empty(F, dtype=torch.float32, device=dev)
        ok = torch.empty(F, dtype=torch.uint8, device=dev)
        slot = torch.empty(F, dtype=torch.int32, device=dev)
        self.decode_into(llr, bits, pm, ok, slot, stream)
        return bits, pm, ok, slot


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


class PolarBatch:
    """Frames of several codes decoded by one persistent launch (batched form).

    codes: list of PolarCode; frame_code: host int array [n_frames] of indices
    into ``codes``; dtype: LLR_F32 or LLR_I8. Inputs / outputs are packed
    buffers laid out by :meth:`layout`.
    """

    def __init__(self, codes, frame_code, dtype=LLR_I8):
        self.codes = list(codes)
        fc = np.ascontiguousarray(np.asarray(frame_code, dtype=np.uint32))
        self.n_frames = int(fc.size)
        self.dtype = int(dtype)
        handles = (ctypes.c_void_p * len(self.codes))(*[c.handle.value for c in self.codes])
        h = ctypes.c_void_p()
        _check(_lib().polar_batch_plan(ctypes.byref(h), ctypes.cast(handles, ctypes.c_void_p), len(self.codes),
                                       fc.ctypes.data_as(ctypes.c_void_p), self.n_frames, self.dtype, 0),
               "polar_batch_plan")
        self._h = h
        self.frame_code = fc

    def close(self):
        if getattr(self, "_h", None):
            _lib().polar_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self):
        """(llr_bytes, bits_bytes, llr_offsets [F] uint64, bits_offsets [F] uint64)."""
        a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
        lo = np.zeros(max(self.n_frames, 1), dtype=np.uint64)
        bo = np.zeros(max(self.n_frames, 1), dtype=np.uint64)
        _check(_lib().polar_batch_layout(self._h, ctypes.byref(a), ctypes.byref(b), lo.ctypes.data_as(ctypes.c_void_p),
                                         bo.ctypes.data_as(ctypes.c_void_p)), "polar_batch_layout")
        return int(a.value), int(b.value), lo[: self.n_frames], bo[: self.n_frames]

    def info(self) -> dict:
        bi = BatchInfo()
        _check(_lib().polar_batch_get_info(self._h, ctypes.byref(bi)), "polar_batch_get_info")
        return {name: int(getattr(bi, name)) for name, _ in BatchInfo._fields_}

    def set_launch(self, warps_per_frame: int, smem_budget: int = 0, cta_threads: int = 0):
        _check(_lib().polar_batch_set_launch(self._h, warps_per_frame, smem_budget, cta_threads),
               "polar_batch_set_launch")

    def run(self, llr, bits, pm, ok=None, slot=None, stream=None):
        _check(_lib().polar_batch_run(self._h, _ptr(llr), _ptr(bits), _ptr(pm), _ptr(ok), _ptr(slot),
                                      _stream_handle(stream)), "polar_batch_run")

    def autotune(self, llr, bits, pm, stream=None):
        w, b, t = ctypes.c_uint32(0), ctypes.c_uint32(0), ctypes.c_uint32(0)
        _check(_lib().polar_batch_autotune(self._h, _ptr(llr), _ptr(bits), _ptr(pm), _stream_handle(stream),
                                           ctypes.byref(w), ctypes.byref(b), ctypes.byref(t)),
               "polar_batch_autotune")
        return int(w.value), int(b.value), int(t.value)

    def capture(self, llr, bits, pm, ok=None, slot=None, stream=None):
        _check(_lib().polar_batch_capture(self._h, _ptr(llr), _ptr(bits), _ptr(pm), _ptr(ok), _ptr(slot),
                                          _stream_handle(stream)), "polar_batch_capture")

    def replay(self, stream=None):
        _check(_lib().polar_batch_replay(self._h, _stream_handle(stream)), "polar_batch_replay")


SERVER_PAUSED = 1


class PolarServer:
    """Continuous-batching decode server (see polar_server_* in include/polar.h)."""

    def __init__(self, device_mem_budget=1 << 30, max_frames_in_flight=1 << 18, warps_per_frame=0,
                 smem_budget=0, paused=False):
        h = ctypes.c_void_p()
        _check(_lib().polar_server_create(ctypes.byref(h), int(device_mem_budget), int(max_frames_in_flight),
                                          int(warps_per_frame), int(smem_budget), SERVER_PAUSED if paused else 0),
               "polar_server_create")
        self._h = h
        self._meta = {}

    def close(self):
        if getattr(self, "_h", None):
            _lib().polar_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, code, llr) -> int:
        """Queue host LLRs ([F, N] float32 or int8 numpy array); returns a ticket."""
        a = np.ascontiguousarray(llr)
        dt = LLR_I8 if a.dtype == np.int8 else LLR_F32
        if dt == LLR_F32:
            a = np.ascontiguousarray(a, dtype=np.float32)
        F = a.size // code.N
        t = ctypes.c_uint64(0)
        _check(_lib().polar_server_submit(self._h, code.handle, a.ctypes.data_as(ctypes.c_void_p), dt, F,
                                          ctypes.byref(t)), "polar_server_submit")
        self._meta[t.value] = (F, (code.k + 7) // 8)
        return int(t.value)

    def poll(self, ticket):
        """None while running, else (bits [F, kb] uint8, penalty [F], crc_ok [F])."""
        F, kb = self._meta[ticket]
        bits = np.zeros((F, kb), dtype=np.uint8)
        pm = np.zeros(F, dtype=np.float32)
        ok = np.zeros(F, dtype=np.uint8)
        done = ctypes.c_int(0)
        _check(_lib().polar_server_poll(self._h, ticket, bits.ctypes.data_as(ctypes.c_void_p),
                                        pm.ctypes.data_as(ctypes.c_void_p), ok.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.byref(done)), "polar_server_poll")
        if not done.value:
            return None
        del self._meta[ticket]
        return bits, pm, ok

    def wait(self, ticket, timeout_ms=60000) -> int:
        """POLAR_OK when done, POLAR_ETIMEDOUT when the bounded wait ran out."""
        return int(_lib().polar_server_wait(self._h, ticket, int(timeout_ms)))

    def result(self, ticket, timeout_ms=60000):
        _check(self.wait(ticket, timeout_ms), "polar_server_wait")
        return self.poll(ticket)

    def pause(self, paused=True):
        _check(_lib().polar_server_pause(self._h, 1 if paused else 0), "polar_server_pause")

    def stats(self, reset=False) -> dict:
        st = ServerStats()
        _check(_lib().polar_server_stats(self._h, ctypes.byref(st), 1 if reset else 0), "polar_server_stats")
        return {name: (getattr(st, name)) for name, _ in ServerStats._fields_}

    def latency(self, min_frames: int, max_frames: int) -> dict:
        """p50 / p99 latency (us) of completed requests of min..max frames."""
        p50, p99, cnt = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
        _check(_lib().polar_server_latency(self._h, min_frames, max_frames, ctypes.byref(p50), ctypes.byref(p99),
                                           ctypes.byref(cnt)), "polar_server_latency")
        return {"p50_us": p50.value, "p99_us": p99.value, "count": cnt.value}
