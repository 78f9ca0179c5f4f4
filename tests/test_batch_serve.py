"""Batched and served solves: the same motif sets as one-at-a-time solves and the oracle.

The mixed batch is 64 planted DNA instances with (l,d) in {(13,4),(15,5),(17,6)}, n in
{10,20,30}, m in {300,600,1000} (some hold ~7e6 motifs).  Every instance is checked three
ways: the batched solve equals the single solve; on the subproblems of the two l-mers of
S_1 at the planted copy (Section 2.3) it equals the stored oracle set; and a sample of its
motifs satisfies the Section 1 predicate directly.  The serving loop (pms_submit /
pms_poll, pms_wait) runs requests that arrive while others are on the GPU, and every
result must equal the same instance solved alone.
"""

from __future__ import annotations

import random
import time

import pytest

import oracle
from conftest import golden_module
from paper_1307_0571_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1307_0571_gb300 import build, pms
    build.build()
    c = pms.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def mix():
    g = golden_module()
    return synth.batched_mix(synth.workload_seed(g.BATCH_SEED_CONFIG, 0), 64)


def test_batched_mix_on_planted_ranges_equals_oracle(ctx, mix):
    from paper_1307_0571_gb300 import pms
    g = golden_module()
    want = g.load_batch()
    assert len(want) == len(mix)
    insts = [pms.Instance(i.seqs, i.n, i.m, "ACGT", i.l, i.d, *g.batch_range(i)) for i in mix]
    got = ctx.solve_batch(insts)
    for i, (a, b) in enumerate(zip(got, want)):
        assert a == b, i
        assert mix[i].motif in a


def test_batched_mix_equals_single_solves_and_is_sound(ctx, mix):
    from paper_1307_0571_gb300 import pms
    batch = ctx.solve_batch([pms.Instance(i.seqs, i.n, i.m, "ACGT", i.l, i.d) for i in mix])
    rng = random.Random(3)
    for inst, got in zip(mix, batch):
        assert got == ctx.solve(inst.seqs, inst.n, inst.m, "ACGT", inst.l, inst.d)
        assert inst.motif in got
        rows = inst.rows()
        for M in rng.sample(got, min(len(got), 20)):
            assert oracle.is_motif(M, rows, inst.d)


def test_serving_results_equal_solves_alone(ctx):
    from paper_1307_0571_gb300 import pms
    stream = synth.serving_stream(synth.workload_seed(5, 0), 24, rate_per_s=40.0)
    t0 = time.time()
    tickets = []
    for arrival, inst in stream:
        while time.time() - t0 < arrival:
            time.sleep(0.001)
        tickets.append(ctx.submit(pms.Instance(inst.seqs, inst.n, inst.m, "ACGT", inst.l,
                                               inst.d)))
    results = {}
    deadline = time.time() + 600
    while len(results) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t not in results:
                r = ctx.poll(t)
                if r is not None:
                    results[t] = r
        time.sleep(0.005)
    assert len(results) == len(tickets)
    for t, (_, inst) in zip(tickets, stream):
        alone = ctx.solve(inst.seqs, inst.n, inst.m, "ACGT", inst.l, inst.d)
        assert results[t] == alone
        assert inst.motif in alone


def test_poll_unknown_ticket(ctx):
    from paper_1307_0571_gb300 import pms
    with pytest.raises(pms.PMSError) as e:
        ctx.poll(10 ** 12)
    assert e.value.code == pms.PMS_E_NOTFOUND


def test_wait_times_out_then_returns_the_result(ctx):
    from paper_1307_0571_gb300 import pms
    inst = synth.planted_instance(synth.workload_seed(2, 1), 20, 600, 17, 6)
    alone = ctx.solve(inst.seqs, 20, 600, "ACGT", 17, 6)   # also tunes the class
    t = ctx.submit(pms.Instance(inst.seqs, 20, 600, "ACGT", 17, 6))
    assert ctx.wait(t, timeout_ms=0) is None     # a (17,6) solve takes ~150 ms
    assert ctx.wait(t) == alone
    with pytest.raises(pms.PMSError) as e:       # the ticket is retired
        ctx.wait(t, timeout_ms=0)
    assert e.value.code == pms.PMS_E_NOTFOUND
    with pytest.raises(pms.PMSError) as e:
        ctx.wait(10 ** 12, timeout_ms=10)
    assert e.value.code == pms.PMS_E_NOTFOUND
