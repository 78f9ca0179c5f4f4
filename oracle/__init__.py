"""Plain CPU oracle for exact planted (l,d) motif search.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA path.

The arithmetic lives in ``pms_oracle.c`` (plain C, one byte per letter); this module only
compiles it with gcc, maps letters to codes and back, and calls it through ctypes.

    hd(u, v)                         Hamming distance (Section 1)
    cd(tuple)                        consensus total distance (Definition 1, Section 2.4)
    theorem1(a, b, c, da, db, dc)    the three-l-mer condition (Theorem 1)
    theorem1_witness(a, b, c, ...)   a common neighbour built as in Theorem 1's proof
    neighborhood(tuple, d, alphabet) common d-neighbourhood by Algorithm 1 (Appendix A)
    is_motif(M, seqs, d)             the motif predicate (Section 1)
    motifs_def(...)                  the motif set by definition (Section 1)
    motifs_pms8(...)                 the motif set by Algorithm 2 (Appendix B)

Parity pins live in tests/test_oracle.py: brute force over all |alphabet|^l l-mers, the
closed-form neighbourhood size, exhaustive Theorem 1 checks, planted-motif recovery and
the invariants of the definition.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pms_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libpmsoracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pms_oracle.c into oracle/_build/libpmsoracle.so with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            lib.oracle_hd.argtypes = [u8p, u8p, ctypes.c_int]
            lib.oracle_cd.argtypes = [u8p, ctypes.c_int, ctypes.c_int]
            lib.oracle_theorem1.argtypes = [u8p, u8p, u8p] + [ctypes.c_int] * 4
            lib.oracle_theorem1_witness.argtypes = [u8p, u8p, u8p] + [ctypes.c_int] * 4 + [u8p]
            lib.oracle_neighborhood.argtypes = [u8p] + [ctypes.c_int] * 4 + [
                ctypes.POINTER(u8p)]
            lib.oracle_neighborhood.restype = ctypes.c_longlong
            lib.oracle_is_motif.argtypes = [u8p, u8p] + [ctypes.c_int] * 4
            lib.oracle_motifs_def.argtypes = [u8p] + [ctypes.c_int] * 8 + [ctypes.POINTER(u8p)]
            lib.oracle_motifs_def.restype = ctypes.c_longlong
            lib.oracle_motifs_pms8.argtypes = [u8p] + [ctypes.c_int] * 9 + [
                ctypes.POINTER(u8p)]
            lib.oracle_motifs_pms8.restype = ctypes.c_longlong
            lib.oracle_free.argtypes = [ctypes.c_void_p]
            _lib = lib
    return _lib


def _codes(s: str, alphabet: str):
    idx = {c: i for i, c in enumerate(alphabet)}
    try:
        b = bytes(idx[c] for c in s)
    except KeyError as e:
        raise ValueError(f"letter {e} is not in the alphabet") from None
    return b, (ctypes.c_uint8 * max(len(b), 1)).from_buffer_copy(b or b"\0")


def _take(lib, ptr, count: int, l: int, alphabet: str) -> list[str]:
    if count < 0:
        raise RuntimeError("oracle failed (bad arguments or out of memory)")
    if count == 0:
        return []
    raw = ctypes.string_at(ptr, count * l)
    lib.oracle_free(ptr)
    table = bytes(ord(c) for c in alphabet) + bytes(256 - len(alphabet))
    txt = raw.translate(table).decode("ascii")
    return [txt[i * l:(i + 1) * l] for i in range(count)]


def hd(u: str, v: str, alphabet: str = "ACGT") -> int:
    lib = _load()
    assert len(u) == len(v)
    return lib.oracle_hd(_codes(u, alphabet)[1], _codes(v, alphabet)[1], len(u))


def cd(tuple_: list[str], alphabet: str = "ACGT") -> int:
    lib = _load()
    l = len(tuple_[0])
    return lib.oracle_cd(_codes("".join(tuple_), alphabet)[1], len(tuple_), l)


def theorem1(a: str, b: str, c: str, da: int, db: int, dc: int,
             alphabet: str = "ACGT") -> bool:
    lib = _load()
    return bool(lib.oracle_theorem1(_codes(a, alphabet)[1], _codes(b, alphabet)[1],
                                    _codes(c, alphabet)[1], len(a), da, db, dc))


def theorem1_witness(a: str, b: str, c: str, da: int, db: int, dc: int,
                     alphabet: str = "ACGT") -> str | None:
    """An l-mer M with Hd(M,a) <= da, Hd(M,b) <= db, Hd(M,c) <= dc, built column by
    column as in the proof of Theorem 1 (Section 2.4); None when the theorem's conditions
    fail (then no such M exists)."""
    lib = _load()
    l = len(a)
    buf = (ctypes.c_uint8 * max(l, 1))()
    ok = lib.oracle_theorem1_witness(_codes(a, alphabet)[1], _codes(b, alphabet)[1],
                                     _codes(c, alphabet)[1], l, da, db, dc, buf)
    return "".join(alphabet[buf[i]] for i in range(l)) if ok else None


def neighborhood(tuple_: list[str], d: int, alphabet: str = "ACGT") -> list[str]:
    lib = _load()
    l = len(tuple_[0])
    out = ctypes.POINTER(ctypes.c_uint8)()
    cnt = lib.oracle_neighborhood(_codes("".join(tuple_), alphabet)[1], len(tuple_), l,
                                  len(alphabet), d, ctypes.byref(out))
    return _take(lib, out, cnt, l, alphabet)


def is_motif(M: str, seqs: list[str], d: int, alphabet: str = "ACGT") -> bool:
    lib = _load()
    m = len(seqs[0])
    return bool(lib.oracle_is_motif(_codes(M, alphabet)[1], _codes("".join(seqs), alphabet)[1],
                                    len(seqs), m, len(M), d))


def _solve(fn, seqs, n, m, alphabet, l, d, extra, x_begin, x_end, threads):
    lib = _load()
    if isinstance(seqs, (list, tuple)):
        seqs = "".join(seqs)
    if isinstance(seqs, (bytes, bytearray)):
        seqs = seqs.decode("ascii")
    if len(seqs) != n * m:
        raise ValueError("seqs must hold n*m letters")
    L = m - l + 1
    xe = L if x_end is None else x_end
    out = ctypes.POINTER(ctypes.c_uint8)()
    args = [_codes(seqs, alphabet)[1], n, m, len(alphabet), l, d] + extra + [
        x_begin, xe, threads, ctypes.byref(out)]
    cnt = getattr(lib, fn)(*args)
    return _take(lib, out, cnt, l, alphabet)


def motifs_def(seqs, n: int, m: int, alphabet: str, l: int, d: int,
               x_begin: int = 0, x_end: int | None = None, threads: int = 0) -> list[str]:
    """Sorted motif set by the definition of Section 1, over candidates from the l-mers
    x_begin..x_end-1 of S_1 (all of them by default).  threads=0 uses every core."""
    return _solve("oracle_motifs_def", seqs, n, m, alphabet, l, d, [], x_begin, x_end,
                  threads)


def motifs_pms8(seqs, n: int, m: int, alphabet: str, l: int, d: int, t: int = 3,
                x_begin: int = 0, x_end: int | None = None, threads: int = 0) -> list[str]:
    """Sorted motif set by Algorithm 2 with threshold stack size t (the set does not
    depend on t)."""
    return _solve("oracle_motifs_pms8", seqs, n, m, alphabet, l, d, [t], x_begin, x_end,
                  threads)
