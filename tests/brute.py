"""Brute force over all |alphabet|^l l-mers, for pinning the oracle on tiny inputs.

Nothing here shares code with the oracle or with the CUDA path: it is the Section 1
definition evaluated for every l-mer of the alphabet at once with numpy.
"""

from __future__ import annotations

import itertools

import numpy as np


def all_lmers(k: int, l: int) -> np.ndarray:
    """Every l-mer over codes 0..k-1, in ascending lexicographic order, shape (k**l, l)."""
    idx = np.arange(k ** l, dtype=np.int64)
    out = np.empty((k ** l, l), dtype=np.int8)
    for p in range(l - 1, -1, -1):
        out[:, p] = idx % k
        idx //= k
    return out


def codes(s: str, alphabet: str) -> np.ndarray:
    return np.array([alphabet.index(c) for c in s], dtype=np.int8)


def to_str(rows: np.ndarray, alphabet: str) -> list[str]:
    return ["".join(alphabet[int(c)] for c in r) for r in rows]


def windows(s: np.ndarray, l: int) -> np.ndarray:
    return np.stack([s[j:j + l] for j in range(len(s) - l + 1)])


def brute_motifs(seqs: list[str], alphabet: str, l: int, d: int) -> list[str]:
    """All M in Sigma^l with, for every string, some window within Hamming distance d."""
    cand = all_lmers(len(alphabet), l)
    keep = np.ones(len(cand), dtype=bool)
    for s in seqs:
        w = windows(codes(s, alphabet), l)
        best = np.full(len(cand), l + 1, dtype=np.int64)
        for j in range(len(w)):
            best = np.minimum(best, (cand != w[j]).sum(axis=1))
        keep &= best <= d
    return to_str(cand[keep], alphabet)


def brute_common_neighbors(tuple_: list[str], budgets: list[int], alphabet: str) -> list[str]:
    """All M with Hd(M, T_i) <= budgets[i] for every i."""
    l = len(tuple_[0])
    cand = all_lmers(len(alphabet), l)
    keep = np.ones(len(cand), dtype=bool)
    for t, b in zip(tuple_, budgets):
        keep &= (cand != codes(t, alphabet)).sum(axis=1) <= b
    return to_str(cand[keep], alphabet)


def min_total_distance(tuple_: list[str], alphabet: str) -> int:
    """min over all M of sum_i Hd(M, T_i)."""
    l = len(tuple_[0])
    cand = all_lmers(len(alphabet), l)
    tot = np.zeros(len(cand), dtype=np.int64)
    for t in tuple_:
        tot += (cand != codes(t, alphabet)).sum(axis=1)
    return int(tot.min())


def column_type_triples(l: int):
    """One canonical DNA triple per multiset of Theorem-1 column types N0..N4 over l columns.

    Column types (Theorem 1's proof): N0 all equal, N1 T1 differs from T2 = T3, N2 T2
    differs from T1 = T3, N3 T3 differs from T1 = T2, N4 all distinct.  Returns
    (a, b, c, counts) with counts = (n0, n1, n2, n3, n4).
    """
    col = {0: ("A", "A", "A"), 1: ("C", "A", "A"), 2: ("A", "C", "A"),
           3: ("A", "A", "C"), 4: ("A", "C", "G")}
    for combo in itertools.combinations_with_replacement(range(5), l):
        a = "".join(col[t][0] for t in combo)
        b = "".join(col[t][1] for t in combo)
        c = "".join(col[t][2] for t in combo)
        counts = tuple(combo.count(t) for t in range(5))
        yield a, b, c, counts
