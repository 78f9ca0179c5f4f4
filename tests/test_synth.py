"""The seeded input generator (paper_1307_0571_gb300/synth.py), which feeds both the CUDA
path and the oracle: SplitMix64 against its published reference outputs, and the planted
instance recipe of Section 1 (exactly d changes per planted copy, at the recorded
position)."""

from __future__ import annotations

import numpy as np
import pytest

from paper_1307_0571_gb300 import synth


def test_splitmix64_reference_outputs():
    # SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) from state 0: its first outputs are
    # the published reference values below.  Output i of the sequence keyed by 0 is the
    # finaliser applied to (i + 1) * gamma.
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    keys = np.array([((i + 1) * synth.GAMMA) & synth.MASK64 for i in range(4)],
                    dtype=np.uint64)
    assert [int(x) for x in synth._mix64(keys)] == want


def test_draws_are_counter_based():
    # any window of a stream equals the same slice of a longer window
    full = synth.draws(7, 3, 0, 100)
    assert np.array_equal(synth.draws(7, 3, 40, 25), full[40:65])
    assert not np.array_equal(synth.draws(7, 4, 0, 100), full)
    assert not np.array_equal(synth.draws(8, 3, 0, 100), full)


@pytest.mark.parametrize("k", [1, 4, 20, 587])
def test_uniform_below_range_and_spread(k):
    x = synth.uniform_below(synth.draws(1, 0, 0, 20000), k)
    assert int(x.min()) >= 0 and int(x.max()) < k
    if k > 1:
        counts = np.bincount(x.astype(np.int64), minlength=k)
        expect = 20000 / k
        assert counts.min() > 0.5 * expect and counts.max() < 1.5 * expect + 5


@pytest.mark.parametrize("alphabet,n,m,l,d", [("ACGT", 20, 600, 17, 6),
                                              (synth.PROTEIN, 8, 100, 15, 7),
                                              ("ACGT", 3, 12, 12, 0),
                                              ("ACGT", 2, 30, 9, 9)])
def test_planted_instance_recipe(alphabet, n, m, l, d):
    inst = synth.planted_instance(123, n, m, l, d, alphabet)
    assert len(inst.seqs) == n * m and set(inst.seqs.decode()) <= set(alphabet)
    assert len(inst.motif) == l and len(inst.positions) == n
    for row, pos in zip(inst.rows(), inst.positions):
        assert 0 <= pos <= m - l
        copy = row[pos:pos + l]
        assert sum(a != b for a, b in zip(copy, inst.motif)) == d
    again = synth.planted_instance(123, n, m, l, d, alphabet)
    assert again.seqs == inst.seqs and again.motif == inst.motif
    assert synth.planted_instance(124, n, m, l, d, alphabet).seqs != inst.seqs


def test_workload_seeds():
    assert synth.workload_seed(2, 0) == 0x504D5338 * 1000 + 200
    assert synth.workload_seed(3, 7) == 0x504D5338 * 1000 + 307
