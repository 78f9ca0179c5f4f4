"""Python binding of libpms (include/pms.h): argument marshalling only.

Every step of the search runs in the library's CUDA kernels.  There is no CPU fallback:
if libpms.so has not been built (``__graft_entry__.build()``) or no sm_103a GPU is
present, the calls raise.

    ctx = Context()                                   # pms_create
    motifs = ctx.solve(seqs, n, m, "ACGT", l, d)      # pms_solve -> sorted list of str
    sets = ctx.solve_batch([Instance(...), ...])      # pms_solve_batch
    count = ctx.solve_device(dseqs_ptr, ..., dout_ptr, cap, stream)   # pms_solve_device
    t = ctx.submit(Instance(...)); ctx.poll(t)        # pms_submit / pms_poll
"""

from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libpms.so")

PMS_OK = 0
PMS_E_INVAL = -1
PMS_E_ALPHABET = -2
PMS_E_NOMEM = -3
PMS_E_OVERFLOW = -4
PMS_E_TIMEOUT = -5
PMS_E_CUDA = -6
PMS_E_BUSY = -7
PMS_E_NOTFOUND = -8

EXPORTS = ["pms_create", "pms_destroy", "pms_solve", "pms_solve_batch", "pms_solve_device",
           "pms_submit", "pms_poll", "pms_wait", "pms_result_free", "pms_strerror",
           "pms_autotune_entries", "pms_autotune_reset", "pms_solve_device_noalloc"]


class pms_opts(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_int), ("warps_per_block", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("max_motifs", ctypes.c_uint64),
                ("mem_budget", ctypes.c_size_t), ("x_begin", ctypes.c_int),
                ("x_end", ctypes.c_int), ("serve_slots", ctypes.c_int),
                ("serve_max_batch", ctypes.c_int)]


class pms_instance(ctypes.Structure):
    _fields_ = [("seqs", ctypes.c_char_p), ("n", ctypes.c_int), ("m", ctypes.c_int),
                ("alphabet", ctypes.c_char_p), ("l", ctypes.c_int), ("d", ctypes.c_int),
                ("x_begin", ctypes.c_int), ("x_end", ctypes.c_int)]


class pms_stats(ctypes.Structure):
    _fields_ = [("items", ctypes.c_uint64), ("tuples", ctypes.c_uint64),
                ("hd_compares", ctypes.c_uint64), ("enum_nodes", ctypes.c_uint64),
                ("leaves", ctypes.c_uint64), ("raw_motifs", ctypes.c_uint64),
                ("cyc_filter", ctypes.c_uint64), ("cyc_enum", ctypes.c_uint64),
                ("cyc_verify", ctypes.c_uint64), ("search_ops", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("busy_max", ctypes.c_uint64),
                ("busy_mean", ctypes.c_uint64), ("item_max", ctypes.c_uint64),
                ("h2d_bytes", ctypes.c_uint64),
                ("d2h_bytes", ctypes.c_uint64), ("kernel_ms", ctypes.c_double),
                ("search_ms", ctypes.c_double),
                ("threshold", ctypes.c_int)]


class pms_result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("l", ctypes.c_int),
                ("motifs", ctypes.c_void_p), ("stats", pms_stats)]


class PMSError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None
_lock = threading.Lock()


def load() -> ctypes.CDLL:
    """Load libpms.so; raises when it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libpms.so is missing ({_LIB_PATH}); build it with "
                               "__graft_entry__.build() or paper_1307_0571_gb300.build")
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        lib.pms_create.argtypes = [P(ctypes.c_void_p), ctypes.c_int, P(pms_opts)]
        lib.pms_destroy.argtypes = [ctypes.c_void_p]
        lib.pms_destroy.restype = None
        lib.pms_solve.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_char_p, ctypes.c_int, ctypes.c_int, P(pms_result)]
        lib.pms_solve_batch.argtypes = [ctypes.c_void_p, P(pms_instance), ctypes.c_int,
                                        P(pms_result)]
        lib.pms_solve_device.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_char_p, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64,
                                         P(ctypes.c_uint64), ctypes.c_void_p, P(pms_stats)]
        lib.pms_submit.argtypes = [ctypes.c_void_p, P(pms_instance), P(ctypes.c_uint64)]
        lib.pms_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, P(pms_result),
                                 P(ctypes.c_int)]
        lib.pms_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint64, P(pms_result), ctypes.c_int]
        lib.pms_result_free.argtypes = [P(pms_result)]
        lib.pms_result_free.restype = None
        lib.pms_strerror.argtypes = [ctypes.c_int]
        lib.pms_strerror.restype = ctypes.c_char_p
        lib.pms_autotune_entries.argtypes = [ctypes.c_void_p]
        lib.pms_autotune_reset.argtypes = [ctypes.c_void_p]
        lib.pms_autotune_reset.restype = None
        lib.pms_solve_device_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_void_p,
                                                 ctypes.c_uint64, P(ctypes.c_uint64),
                                                 ctypes.c_void_p]
        _lib = lib
        return lib


def solve_device_noalloc(d_seqs: int, n: int, m: int, alphabet: str, l: int, d: int,
                         d_motifs: int, cap: int, stream: int = 0, threshold: int = 0) -> int:
    """pms_solve_device_noalloc: the device-resident solve using only the library's fixed
    scratch array (for callers that must not allocate device memory while running).
    Returns the motif count; the motifs are in d_motifs."""
    lib = load()
    cnt = ctypes.c_uint64(0)
    rc = lib.pms_solve_device_noalloc(ctypes.c_void_p(d_seqs), n, m, alphabet.encode("ascii"),
                                      l, d, threshold, ctypes.c_void_p(d_motifs), cap,
                                      ctypes.byref(cnt), ctypes.c_void_p(stream))
    if rc != PMS_OK:
        raise PMSError(rc, "pms_solve_device_noalloc")
    return cnt.value


def strerror(code: int) -> str:
    return load().pms_strerror(code).decode()


@dataclass
class Instance:
    seqs: bytes
    n: int
    m: int
    alphabet: str
    l: int
    d: int
    x_begin: int = 0        # subproblems of l-mers x_begin..x_end-1 of S_1; 0, 0 = all
    x_end: int = 0


def _b(x) -> bytes:
    if isinstance(x, str):
        return x.encode("ascii")
    if isinstance(x, (list, tuple)):
        return "".join(x).encode("ascii")
    return bytes(x)


def _take(lib, res: pms_result) -> list[str]:
    try:
        if res.count == 0:
            return []
        raw = ctypes.string_at(res.motifs, res.count * res.l).decode("ascii")
        return [raw[i * res.l:(i + 1) * res.l] for i in range(res.count)]
    finally:
        lib.pms_result_free(ctypes.byref(res))


class Context:
    """A pms_ctx on one CUDA device."""

    def __init__(self, device: int = 0, **opts):
        self.lib = load()
        o = pms_opts()
        for k, v in opts.items():
            setattr(o, k, v)
        self.opts = o
        h = ctypes.c_void_p()
        rc = self.lib.pms_create(ctypes.byref(h), device, ctypes.byref(o))
        if rc != PMS_OK:
            raise PMSError(rc, "pms_create")
        self.h = h
        self.last_stats: pms_stats | None = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.pms_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, seqs, n: int, m: int, alphabet: str, l: int, d: int) -> list[str]:
        res = pms_result()
        rc = self.lib.pms_solve(self.h, _b(seqs), n, m, alphabet.encode("ascii"), l, d,
                                ctypes.byref(res))
        if rc != PMS_OK:
            raise PMSError(rc, "pms_solve")
        self.last_stats = pms_stats.from_buffer_copy(res.stats)
        return _take(self.lib, res)

    def solve_ptr(self, host_ptr: int, n: int, m: int, alphabet: str, l: int, d: int) -> list[str]:
        """pms_solve on sequences at a host address (e.g. pinned memory)."""
        res = pms_result()
        rc = self.lib.pms_solve(self.h, ctypes.cast(ctypes.c_void_p(host_ptr), ctypes.c_char_p),
                                n, m, alphabet.encode("ascii"), l, d, ctypes.byref(res))
        if rc != PMS_OK:
            raise PMSError(rc, "pms_solve")
        self.last_stats = pms_stats.from_buffer_copy(res.stats)
        return _take(self.lib, res)

    def solve_batch(self, insts: list[Instance]) -> list[list[str]]:
        arr = (pms_instance * len(insts))()
        keep = []
        for i, it in enumerate(insts):
            s, a = _b(it.seqs), it.alphabet.encode("ascii")
            keep += [s, a]
            arr[i] = pms_instance(s, it.n, it.m, a, it.l, it.d, it.x_begin, it.x_end)
        outs = (pms_result * len(insts))()
        rc = self.lib.pms_solve_batch(self.h, arr, len(insts), outs)
        if rc != PMS_OK:
            raise PMSError(rc, "pms_solve_batch")
        if len(insts):
            self.last_stats = pms_stats.from_buffer_copy(outs[0].stats)
        return [_take(self.lib, outs[i]) for i in range(len(insts))]

    def solve_device(self, d_seqs: int, n: int, m: int, alphabet: str, l: int, d: int,
                     d_motifs: int, cap: int, stream: int = 0) -> tuple[int, pms_stats]:
        """Device pointers in, device pointer out; returns (count, stats)."""
        cnt = ctypes.c_uint64(0)
        st = pms_stats()
        rc = self.lib.pms_solve_device(self.h, ctypes.c_void_p(d_seqs), n, m,
                                       alphabet.encode("ascii"), l, d,
                                       ctypes.c_void_p(d_motifs), cap, ctypes.byref(cnt),
                                       ctypes.c_void_p(stream), ctypes.byref(st))
        if rc != PMS_OK:
            raise PMSError(rc, "pms_solve_device")
        self.last_stats = st
        return cnt.value, st

    def submit(self, it: Instance) -> int:
        s, a = _b(it.seqs), it.alphabet.encode("ascii")
        inst = pms_instance(s, it.n, it.m, a, it.l, it.d, it.x_begin, it.x_end)
        t = ctypes.c_uint64(0)
        rc = self.lib.pms_submit(self.h, ctypes.byref(inst), ctypes.byref(t))
        if rc != PMS_OK:
            raise PMSError(rc, "pms_submit")
        return t.value

    def poll(self, ticket: int):
        """None while pending, else the sorted motif list."""
        res = pms_result()
        done = ctypes.c_int(0)
        rc = self.lib.pms_poll(self.h, ticket, ctypes.byref(res), ctypes.byref(done))
        if not done.value:
            if rc != PMS_OK:
                raise PMSError(rc, "pms_poll")
            return None
        if rc != PMS_OK:
            self.lib.pms_result_free(ctypes.byref(res))
            raise PMSError(rc, "pms_poll")
        return _take(self.lib, res)

    def wait(self, ticket: int, timeout_ms: int = -1):
        """The sorted motif list once the ticket finishes; None if timeout_ms passes first
        (negative: wait without limit)."""
        res = pms_result()
        rc = self.lib.pms_wait(self.h, ticket, ctypes.byref(res), int(timeout_ms))
        if rc == PMS_E_TIMEOUT:
            return None
        if rc != PMS_OK:
            self.lib.pms_result_free(ctypes.byref(res))
            raise PMSError(rc, "pms_wait")
        return _take(self.lib, res)

    def autotune_entries(self) -> int:
        return self.lib.pms_autotune_entries(self.h)
