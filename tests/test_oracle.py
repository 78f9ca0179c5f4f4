"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: brute force over all
|alphabet|^l l-mers, closed forms (the neighbourhood size of Appendix C/D, Cd identities of
Theorem 1's proof), the exhaustive truth table of Theorem 1, recovery of the planted motif,
and invariants of the Section 1 definition.
"""

from __future__ import annotations

import itertools
import random
from math import comb

import numpy as np
import pytest

import brute
from paper_1307_0571_gb300 import synth


def _rand_seqs(rng, n, m, alphabet):
    return ["".join(rng.choice(alphabet) for _ in range(m)) for _ in range(n)]


def _n_d(l, d, k):
    """N_d = sum_{i=0}^{d} C(l,i) (k-1)^i (Appendix D; the Appendix C form is garbled)."""
    return sum(comb(l, i) * (k - 1) ** i for i in range(0, min(d, l) + 1))


# ------------------------------------------------------------------ basic distances

def test_hd_examples(oracle_lib):
    assert oracle_lib.hd("ACGT", "ACGT") == 0
    assert oracle_lib.hd("ACGT", "TGCA") == 4
    assert oracle_lib.hd("AACCGGTT", "AACCGGTA") == 1


def test_cd_equals_hd_for_two(oracle_lib):
    # Section 2.4: Cd(A,B) = Hd(A,B)
    rng = random.Random(1)
    for _ in range(200):
        l = rng.randint(1, 12)
        a = "".join(rng.choice("ACGT") for _ in range(l))
        b = "".join(rng.choice("ACGT") for _ in range(l))
        assert oracle_lib.cd([a, b]) == oracle_lib.hd(a, b)


def test_cd_three_by_column_types(oracle_lib):
    # Theorem 1's proof: for three l-mers Cd = n1 + n2 + n3 + 2 n4, and
    # Hd(T_i, T_j) = n_i + n_j + n4.
    for l in range(1, 6):
        for a, b, c, (n0, n1, n2, n3, n4) in brute.column_type_triples(l):
            assert oracle_lib.cd([a, b, c]) == n1 + n2 + n3 + 2 * n4
            assert oracle_lib.hd(a, b) == n1 + n2 + n4
            assert oracle_lib.hd(a, c) == n1 + n3 + n4
            assert oracle_lib.hd(b, c) == n2 + n3 + n4


@pytest.mark.parametrize("k,alphabet", [(4, "ACGT"), (3, "ABC"), (5, "ABCDE")])
def test_cd_is_min_total_distance(oracle_lib, k, alphabet):
    # Cd(T) is a lower bound on sum_i Hd(M, T_i) (Section 2.4) and the column-wise majority
    # letter attains it, so Cd(T) = min_M sum_i Hd(M, T_i).
    rng = random.Random(2)
    for _ in range(40):
        l = rng.randint(1, 5)
        t = rng.randint(1, 6)
        tup = ["".join(rng.choice(alphabet) for _ in range(l)) for _ in range(t)]
        assert oracle_lib.cd(tup, alphabet) == brute.min_total_distance(tup, alphabet)


# --------------------------------------------------------------------- Theorem 1

def _exists(a, b, c, da, db, dc, alphabet):
    return len(brute.brute_common_neighbors([a, b, c], [da, db, dc], alphabet)) > 0


@pytest.mark.parametrize("l", [1, 2, 3, 4, 5])
def test_theorem1_exhaustive_column_types(oracle_lib, l):
    # The existence of a common neighbour depends only on the counts of column types
    # N0..N4 (columns are independent), so one canonical triple per multiset, with every
    # budget triple in [0, l]^3 (and -1), covers every DNA triple of length l.
    for a, b, c, _ in brute.column_type_triples(l):
        cand = brute.all_lmers(4, l)
        dist = [(cand != brute.codes(s, "ACGT")).sum(axis=1) for s in (a, b, c)]
        for da, db, dc in itertools.product(range(-1, l + 1), repeat=3):
            truth = bool(((dist[0] <= da) & (dist[1] <= db) & (dist[2] <= dc)).any())
            assert oracle_lib.theorem1(a, b, c, da, db, dc) == truth, (a, b, c, da, db, dc)


@pytest.mark.parametrize("alphabet", ["ACGT", "ACDEFGHIKLMNPQRSTVWY", "AB"])
def test_theorem1_random_triples(oracle_lib, alphabet):
    rng = random.Random(3)
    k = len(alphabet)
    lmax = {2: 10, 4: 7, 20: 3}[k]
    for _ in range(150):
        l = rng.randint(1, lmax)
        a, b, c = ("".join(rng.choice(alphabet) for _ in range(l)) for _ in range(3))
        da, db, dc = (rng.randint(0, l) for _ in range(3))
        assert oracle_lib.theorem1(a, b, c, da, db, dc, alphabet) == _exists(
            a, b, c, da, db, dc, alphabet)


def _hd(u, v):
    return sum(x != y for x, y in zip(u, v))


@pytest.mark.parametrize("l", [1, 2, 3, 4, 5])
def test_theorem1_witness_exhaustive_column_types(oracle_lib, l):
    # The construction in the proof of Theorem 1 yields a common neighbour exactly when
    # one exists (brute force over all 4^l l-mers), for every column-type multiset.
    for a, b, c, _ in brute.column_type_triples(l):
        cand = brute.all_lmers(4, l)
        dist = [(cand != brute.codes(s, "ACGT")).sum(axis=1) for s in (a, b, c)]
        for da, db, dc in itertools.product(range(0, l + 1), repeat=3):
            truth = bool(((dist[0] <= da) & (dist[1] <= db) & (dist[2] <= dc)).any())
            M = oracle_lib.theorem1_witness(a, b, c, da, db, dc)
            assert (M is not None) == truth, (a, b, c, da, db, dc)
            if M is not None:
                assert _hd(M, a) <= da and _hd(M, b) <= db and _hd(M, c) <= dc


@pytest.mark.parametrize("alphabet", ["ACGT", "ACDEFGHIKLMNPQRSTVWY"])
def test_theorem1_witness_long_lmers(oracle_lib, alphabet):
    # At lengths brute force cannot reach: triples planted around a random M0 (so a common
    # neighbour exists and the witness must be one), and random triples with budgets near
    # the pair limits (the witness exists exactly when the conditions of Theorem 1 hold,
    # and then it is a common neighbour).  Both cases of the proof occur.
    rng = random.Random(11)
    for _ in range(300):
        l = rng.randint(15, 64)
        m0 = [rng.choice(alphabet) for _ in range(l)]
        trip, budgets = [], []
        for _ in range(3):
            di = rng.randint(0, l // 2)
            s = list(m0)
            for pos in rng.sample(range(l), di):
                s[pos] = rng.choice([x for x in alphabet if x != m0[pos]])
            trip.append("".join(s))
            budgets.append(di)
        M = oracle_lib.theorem1_witness(*trip, *budgets, alphabet)
        assert M is not None
        assert all(_hd(M, t) <= di for t, di in zip(trip, budgets))
    for _ in range(300):
        l = rng.randint(15, 64)
        a, b, c = ("".join(rng.choice(alphabet) for _ in range(l)) for _ in range(3))
        hab, hac, hbc = _hd(a, b), _hd(a, c), _hd(b, c)
        da = rng.randint(0, l)
        db = max(0, hab - da + rng.randint(-2, 2))
        dc = max(0, max(hac - da, hbc - db) + rng.randint(-2, 2))
        M = oracle_lib.theorem1_witness(a, b, c, da, db, dc, alphabet)
        assert (M is not None) == oracle_lib.theorem1(a, b, c, da, db, dc, alphabet)
        if M is not None:
            assert _hd(M, a) <= da and _hd(M, b) <= db and _hd(M, c) <= dc


# ---------------------------------------------------------------- Algorithm 1

@pytest.mark.parametrize("l,d,alphabet", [(5, 0, "ACGT"), (6, 2, "ACGT"), (8, 3, "ACGT"),
                                          (10, 4, "ACGT"), (4, 2, "ACDEFGHIKLMNPQRSTVWY"),
                                          (7, 7, "AB"), (3, 5, "ACG")])
def test_neighborhood_size_closed_form(oracle_lib, l, d, alphabet):
    # |d-neighbourhood of one l-mer| = sum_{i<=d} C(l,i)(|Sigma|-1)^i (Appendix D).
    rng = random.Random(l * 31 + d)
    x = "".join(rng.choice(alphabet) for _ in range(l))
    nb = oracle_lib.neighborhood([x], d, alphabet)
    assert len(nb) == _n_d(l, d, len(alphabet))
    assert len(set(nb)) == len(nb)
    assert nb == sorted(nb, key=lambda s: [alphabet.index(c) for c in s])
    if l <= 8:
        assert nb == brute.brute_common_neighbors([x], [d], alphabet)


@pytest.mark.parametrize("t", [2, 3, 4, 5])
def test_neighborhood_tuples_vs_brute(oracle_lib, t):
    rng = random.Random(10 + t)
    for _ in range(25):
        l = rng.randint(3, 8)
        d = rng.randint(0, l // 2 + 1)
        base = "".join(rng.choice("ACGT") for _ in range(l))
        tup = []
        for _ in range(t):   # l-mers near a common centre, so neighbourhoods are non-empty
            s = list(base)
            for p in rng.sample(range(l), rng.randint(0, d + 1)):
                s[p] = rng.choice("ACGT")
            tup.append("".join(s))
        assert oracle_lib.neighborhood(tup, d) == brute.brute_common_neighbors(
            tup, [d] * t, "ACGT")


# ------------------------------------------------------- motif sets vs brute force

def _tiny_cases():
    rng = random.Random(4)
    cases = []
    for _ in range(18):
        alphabet = rng.choice(["ACGT", "ACGT", "ACGT", "ABC", "AB"])
        l = rng.randint(2, 7 if len(alphabet) == 4 else 8)
        d = rng.randint(0, max(0, l // 2))
        n = rng.randint(1, 6)
        m = rng.randint(l, 30)
        cases.append((alphabet, l, d, n, m, rng.randint(0, 10 ** 9)))
    cases.append(("ACDEFGHIKLMNPQRSTVWY", 3, 1, 3, 20, 5))
    cases.append(("ACDEFGHIKLMNPQRSTVWY", 2, 1, 4, 12, 6))
    return cases


@pytest.mark.parametrize("alphabet,l,d,n,m,seed", _tiny_cases())
def test_motif_sets_vs_brute_force(oracle_lib, alphabet, l, d, n, m, seed):
    rng = random.Random(seed)
    seqs = _rand_seqs(rng, n, m, alphabet)
    truth = brute.brute_motifs(seqs, alphabet, l, d)
    assert oracle_lib.motifs_def(seqs, n, m, alphabet, l, d) == truth
    for t in (1, 2, 3, n + 1):
        assert oracle_lib.motifs_pms8(seqs, n, m, alphabet, l, d, t=t) == truth


@pytest.mark.parametrize("seed", range(6))
def test_planted_tiny_vs_brute_force(oracle_lib, seed):
    inst = synth.planted_instance(seed, 6, 40, 8, 2)
    truth = brute.brute_motifs(inst.rows(), "ACGT", 8, 2)
    assert inst.motif in truth
    assert oracle_lib.motifs_def(inst.seqs, 6, 40, "ACGT", 8, 2) == truth
    assert oracle_lib.motifs_pms8(inst.seqs, 6, 40, "ACGT", 8, 2, t=2) == truth


# ------------------------------------------------ definition-level invariants

def _inst(seed, n=8, m=80, l=9, d=2, alphabet="ACGT"):
    return synth.planted_instance(seed, n, m, l, d, alphabet)


@pytest.mark.parametrize("seed", range(4))
def test_pms8_equals_definition_medium(oracle_lib, seed):
    inst = _inst(100 + seed, n=10, m=120, l=10, d=3)
    a = oracle_lib.motifs_def(inst.seqs, inst.n, inst.m, "ACGT", inst.l, inst.d)
    assert inst.motif in a
    for t in (1, 2, 3, 4, 11):
        assert oracle_lib.motifs_pms8(inst.seqs, inst.n, inst.m, "ACGT", inst.l, inst.d,
                                      t=t) == a


def test_order_of_strings_does_not_matter(oracle_lib):
    inst = _inst(7, n=8, m=60, l=8, d=2)
    rows = inst.rows()
    base = oracle_lib.motifs_def(rows, 8, 60, "ACGT", 8, 2)
    rng = random.Random(5)
    for _ in range(3):
        perm = rows[:]
        rng.shuffle(perm)
        assert oracle_lib.motifs_def(perm, 8, 60, "ACGT", 8, 2) == base
        assert oracle_lib.motifs_pms8(perm, 8, 60, "ACGT", 8, 2, t=3) == base


def test_alphabet_relabelling(oracle_lib):
    inst = _inst(8, n=6, m=50, l=7, d=2)
    base = oracle_lib.motifs_def(inst.seqs, 6, 50, "ACGT", 7, 2)
    relabel = str.maketrans("ACGT", "TGCA")
    seqs2 = inst.seqs.decode().translate(relabel)
    got = oracle_lib.motifs_def(seqs2, 6, 50, "ACGT", 7, 2)
    assert got == sorted(s.translate(relabel) for s in base)
    # the same strings read in another alphabet order give the same set, in that order
    got2 = oracle_lib.motifs_def(inst.seqs, 6, 50, "TGCA", 7, 2)
    assert sorted(got2) == sorted(base)
    assert got2 == sorted(base, key=lambda s: ["TGCA".index(c) for c in s])


def test_reversal(oracle_lib):
    inst = _inst(9, n=6, m=50, l=8, d=2)
    base = oracle_lib.motifs_def(inst.seqs, 6, 50, "ACGT", 8, 2)
    rev = [r[::-1] for r in inst.rows()]
    got = oracle_lib.motifs_def(rev, 6, 50, "ACGT", 8, 2)
    assert got == sorted(s[::-1] for s in base)


def test_monotone_in_d(oracle_lib):
    inst = _inst(10, n=6, m=40, l=8, d=1)
    prev = set()
    for d in range(0, 5):
        cur = set(oracle_lib.motifs_def(inst.seqs, 6, 40, "ACGT", 8, d))
        assert prev <= cur
        prev = cur


def test_d_zero_is_intersection(oracle_lib):
    inst = synth.random_instance(11, 5, 200, 4, 0)
    rows = inst.rows()
    sets = [set(r[j:j + 4] for j in range(200 - 4 + 1)) for r in rows]
    truth = sorted(set.intersection(*sets))
    assert oracle_lib.motifs_def(rows, 5, 200, "ACGT", 4, 0) == truth
    assert oracle_lib.motifs_pms8(rows, 5, 200, "ACGT", 4, 0, t=2) == truth


def test_single_string_is_union_of_neighbourhoods(oracle_lib):
    s = "ACGTTGCAAC"
    l, d = 5, 1
    union = set()
    for j in range(len(s) - l + 1):
        x = s[j:j + l]
        for p in range(l):
            for c in "ACGT":
                union.add(x[:p] + c + x[p + 1:])
    assert oracle_lib.motifs_def([s], 1, len(s), "ACGT", l, d) == sorted(union)
    assert oracle_lib.motifs_pms8([s], 1, len(s), "ACGT", l, d, t=1) == sorted(union)


def test_d_at_least_l_gives_everything(oracle_lib):
    seqs = ["ACG", "TTA"]
    got = oracle_lib.motifs_def(seqs, 2, 3, "ACGT", 2, 2)
    assert got == ["".join(p) for p in itertools.product("ACGT", repeat=2)]


def test_x_ranges_merge_to_whole(oracle_lib):
    # Section 2.3: the subproblems of the l-mers of S_1 are independent; a split of the
    # range of x, merged, gives the whole set.
    inst = _inst(12, n=8, m=70, l=9, d=2)
    L = 70 - 9 + 1
    whole = oracle_lib.motifs_def(inst.seqs, 8, 70, "ACGT", 9, 2)
    parts = set()
    for a, b in [(0, 17), (17, 40), (40, L)]:
        parts |= set(oracle_lib.motifs_pms8(inst.seqs, 8, 70, "ACGT", 9, 2, t=2,
                                            x_begin=a, x_end=b))
    assert sorted(parts) == whole


def test_is_motif_matches_brute(oracle_lib):
    rng = random.Random(13)
    seqs = _rand_seqs(rng, 4, 25, "ACGT")
    truth = set(brute.brute_motifs(seqs, "ACGT", 6, 2))
    for M in brute.to_str(brute.all_lmers(4, 6)[::37], "ACGT"):
        assert oracle_lib.is_motif(M, seqs, 2) == (M in truth)


# ---------------------------------------------------------- planted recovery

@pytest.mark.parametrize("seed", range(5))
def test_planted_motif_recovered(oracle_lib, seed):
    # Section 1 instances: every planted copy is within d of the motif, so it is a motif.
    inst = synth.planted_instance(synth.workload_seed(9, seed), 20, 300, 11, 3)
    got = oracle_lib.motifs_pms8(inst.seqs, 20, 300, "ACGT", 11, 3, t=2)
    assert inst.motif in got
    for M in got:
        assert oracle_lib.is_motif(M, inst.rows(), 3)


def test_planted_protein(oracle_lib):
    inst = synth.planted_instance(5, 6, 40, 5, 1, synth.PROTEIN)
    got = oracle_lib.motifs_pms8(inst.seqs, 6, 40, synth.PROTEIN, 5, 1, t=2)
    assert inst.motif in got
    assert got == oracle_lib.motifs_def(inst.seqs, 6, 40, synth.PROTEIN, 5, 1)


# ------------------------------------------------ expected spurious count (App. C)

def test_spurious_count_matches_estimate(oracle_lib):
    # Appendix C: E[#motifs of a random instance] = |S|^l q^n with
    # q = 1 - (1 - N_d/|S|^l)^(m-l+1).  A statistical check over 40 random instances.
    l, d, n, m = 8, 2, 4, 30
    k = 4
    q = 1 - (1 - _n_d(l, d, k) / k ** l) ** (m - l + 1)
    expect = k ** l * q ** n
    counts = []
    for s in range(40):
        inst = synth.random_instance(1000 + s, n, m, l, d)
        counts.append(len(oracle_lib.motifs_def(inst.seqs, n, m, "ACGT", l, d)))
    mean = float(np.mean(counts))
    assert 0.6 * expect < mean < 1.4 * expect, (mean, expect)


def test_bad_arguments_raise(oracle_lib):
    with pytest.raises(RuntimeError):
        oracle_lib.motifs_def("ACGT", 1, 4, "ACGT", 5, 1)     # l > m
    with pytest.raises(ValueError):
        oracle_lib.motifs_def("ACGX", 1, 4, "ACGT", 2, 1)     # letter not in alphabet
