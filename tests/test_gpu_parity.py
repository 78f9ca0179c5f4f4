"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Motif sets are integer/string results, so the bar is bit-exact equality of the sorted
sets.  Small cases run the definition oracle directly; instances of the paper's size use
the PMS8 oracle (pinned to the definition in test_oracle.py) or stored golden sets written
by tests/golden/make_golden.py from the oracle alone.
"""

from __future__ import annotations

import random

import pytest

import oracle
from paper_1307_0571_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1307_0571_gb300 import build, pms
    build.build()
    c = pms.Context(0)
    yield c
    c.close()


def _ctx(**kw):
    from paper_1307_0571_gb300 import pms
    return pms.Context(0, **kw)


def _small_cases():
    rng = random.Random(77)
    cases = []
    for _ in range(14):
        l = rng.randint(5, 12)
        d = rng.randint(0, max(1, l // 3))
        n = rng.randint(2, 9)
        m = rng.randint(l, 90)
        cases.append((l, d, n, m, rng.randint(0, 10 ** 6)))
    cases += [(8, 2, 1, 30, 1), (9, 2, 2, 40, 2), (7, 7, 2, 9, 3), (6, 0, 5, 50, 4),
              (10, 3, 20, 10, 5), (12, 3, 64, 40, 6), (9, 2, 7, 9, 7)]
    return cases


@pytest.mark.parametrize("l,d,n,m,seed", _small_cases())
def test_small_random_vs_definition(ctx, l, d, n, m, seed):
    inst = synth.planted_instance(seed, n, m, l, d)
    want = oracle.motifs_def(inst.seqs, n, m, "ACGT", l, d)
    got = ctx.solve(inst.seqs, n, m, "ACGT", l, d)
    assert got == want


@pytest.mark.parametrize("t", [2, 3, 4, 5, 8])
def test_threshold_does_not_change_the_set(t):
    inst = synth.planted_instance(31, 12, 160, 11, 3)
    want = oracle.motifs_def(inst.seqs, 12, 160, "ACGT", 11, 3)
    with _ctx(threshold=t) as c:
        assert c.solve(inst.seqs, 12, 160, "ACGT", 11, 3) == want


@pytest.mark.parametrize("seed", range(2))
def test_13_4_full_size(ctx, seed):
    inst = synth.planted_instance(synth.workload_seed(1, seed), 20, 600, 13, 4)
    want = oracle.motifs_pms8(inst.seqs, 20, 600, "ACGT", 13, 4, t=2)
    got = ctx.solve(inst.seqs, 20, 600, "ACGT", 13, 4)
    assert inst.motif in got
    assert got == want


def test_protein_small(ctx):
    inst = synth.planted_instance(5, 6, 60, 6, 2, synth.PROTEIN)
    want = oracle.motifs_def(inst.seqs, 6, 60, synth.PROTEIN, 6, 2)
    assert ctx.solve(inst.seqs, 6, 60, synth.PROTEIN, 6, 2) == want


def test_long_l_two_words(ctx):
    inst = synth.planted_instance(8, 8, 120, 40, 6)
    want = oracle.motifs_pms8(inst.seqs, 8, 120, "ACGT", 40, 6, t=3)
    got = ctx.solve(inst.seqs, 8, 120, "ACGT", 40, 6)
    assert inst.motif in got
    assert got == want


_LONG_L = {}


def _long_l_case(l, d, n, m):
    """DNA l-mers longer than 32 letters (two-word planes) with a many-motif answer."""
    key = (l, d, n, m)
    if key not in _LONG_L:
        inst = synth.planted_instance(78, n, m, l, d)
        _LONG_L[key] = (inst, oracle.motifs_pms8(inst.seqs, n, m, "ACGT", l, d, t=4))
    return _LONG_L[key]


@pytest.mark.parametrize("l,d,n,m", [(34, 12, 6, 50), (36, 13, 6, 60)])
@pytest.mark.parametrize("t", [4, 5, 6])
def test_long_l_thresholds(l, d, n, m, t):
    # (threshold 3 is left out: common d-neighbourhoods of three such l-mers hold ~1e10
    # l-mers, out of reach for any implementation of Algorithm 1)
    inst, want = _long_l_case(l, d, n, m)
    assert inst.motif in want and len(want) > 10
    with _ctx(threshold=t) as c:
        assert c.solve(inst.seqs, n, m, "ACGT", l, d) == want


_A32 = "ABCDEFGHIJKLMNOPQRSTUVWXYZ012345"


@pytest.mark.parametrize("n,m,l,d,alphabet,seed", [
    (5, 70, 64, 3, "ACGT", 11),              # longest DNA l-mers (two 32-bit words a plane)
    (4, 40, 25, 2, synth.PROTEIN, 12),       # longest l for 20 letters (5 bits a letter)
    (4, 40, 5, 2, _A32, 13),                 # the largest alphabet
    (4, 40, 25, 1, _A32, 14),                # largest alphabet at its longest l
])
def test_size_limits_vs_definition(ctx, n, m, l, d, alphabet, seed):
    inst = synth.planted_instance(seed, n, m, l, d, alphabet)
    want = oracle.motifs_def(inst.seqs, n, m, alphabet, l, d)
    assert inst.motif in want
    assert ctx.solve(inst.seqs, n, m, alphabet, l, d) == want


def test_beyond_size_limits(ctx):
    from paper_1307_0571_gb300 import pms
    dna = synth.random_instance(3, 2, 80, 65, 3)
    prot = synth.random_instance(3, 2, 40, 26, 3, synth.PROTEIN)
    for args in [(dna.seqs, 2, 80, "ACGT", 65, 3),                      # l > 64
                 (prot.seqs, 2, 40, synth.PROTEIN, 26, 3),              # 5 * 26 bits > 128
                 (b"AC" * 65, 65, 2, "ACGT", 2, 0),                     # n > 64
                 (b"ACGT", 1, 4, "A", 2, 0),                            # one-letter alphabet
                 (b"A" * 8, 1, 8, "".join(chr(48 + i) for i in range(33)), 2, 0)]:
        with pytest.raises(pms.PMSError) as e:
            ctx.solve(*args)
        assert e.value.code == pms.PMS_E_INVAL, args[3:]


def test_batch_equals_single(ctx):
    from paper_1307_0571_gb300 import pms
    insts = [synth.planted_instance(40 + i, 5 + i, 60 + 13 * i, 8 + (i % 3), 2)
             for i in range(7)]
    batch = ctx.solve_batch([pms.Instance(i.seqs, i.n, i.m, "ACGT", i.l, i.d) for i in insts])
    for inst, got in zip(insts, batch):
        assert got == oracle.motifs_def(inst.seqs, inst.n, inst.m, "ACGT", inst.l, inst.d)


def test_alphabet_error(ctx):
    from paper_1307_0571_gb300 import pms
    with pytest.raises(pms.PMSError) as e:
        ctx.solve(b"ACGTN" * 4, 2, 10, "ACGT", 4, 1)
    assert e.value.code == pms.PMS_E_ALPHABET


def test_invalid_sizes(ctx):
    from paper_1307_0571_gb300 import pms
    for args in [(b"ACGT", 1, 4, "ACGT", 5, 1), (b"ACGT", 1, 4, "AC", 2, -1),
                 (b"ACGT", 1, 4, "AAC", 2, 1)]:
        with pytest.raises(pms.PMSError) as e:
            ctx.solve(*args)
        assert e.value.code == pms.PMS_E_INVAL


def test_solve_device(ctx):
    import torch
    inst = synth.planted_instance(9, 10, 150, 10, 2)
    want = oracle.motifs_def(inst.seqs, 10, 150, "ACGT", 10, 2)
    dseq = torch.frombuffer(bytearray(inst.seqs), dtype=torch.uint8).cuda()
    cap = 1000
    dout = torch.empty(cap * 10, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    count, st = ctx.solve_device(dseq.data_ptr(), 10, 150, "ACGT", 10, 2, dout.data_ptr(), cap,
                                 s.cuda_stream)
    raw = bytes(dout[:count * 10].cpu().numpy().tobytes()).decode()
    assert [raw[i * 10:(i + 1) * 10] for i in range(count)] == want
