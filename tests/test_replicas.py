"""Replica sharding and merge on CPU with gloo, world_size 2 (no GPU).

Each rank solves its range of l-mers of S_1 (Section 2.3) with the CPU oracle standing in
for its GPU, the ranks all-gather their sorted sets, and the merge must equal the whole
set computed in one piece.
"""

from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1307_0571_gb300.replicas import merge_sorted, shard_ranges


def test_shard_ranges_cover_exactly():
    for L in (1, 7, 584, 1000):
        for w in (1, 2, 3, 8):
            r = shard_ranges(L, w)
            assert r[0][0] == 0 and r[-1][1] == L
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [hi - lo for lo, hi in r]
            assert max(sizes) - min(sizes) <= 1


def test_merge_sorted_orders_and_dedupes():
    assert merge_sorted([["AC", "GT"], ["AC", "CA", "TT"]], "ACGT") == ["AC", "CA", "GT", "TT"]
    assert merge_sorted([["TG", "GA"], ["GG"]], "TGCA") == ["TG", "GG", "GA"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1307_0571_gb300 import synth
    from paper_1307_0571_gb300.replicas import solve_sharded
    inst = synth.planted_instance(314, 8, 90, 10, 2)
    L = inst.m - inst.l + 1
    got = solve_sharded(lambda a, b: oracle.motifs_pms8(inst.seqs, inst.n, inst.m, "ACGT",
                                                        inst.l, inst.d, t=3, x_begin=a,
                                                        x_end=b, threads=1),
                        L, "ACGT", rank, world)
    q.put((rank, got))
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_whole_set():
    import oracle
    from paper_1307_0571_gb300 import synth
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    inst = synth.planted_instance(314, 8, 90, 10, 2)
    whole = oracle.motifs_def(inst.seqs, inst.n, inst.m, "ACGT", inst.l, inst.d)
    assert inst.motif in whole
    assert results[0] == results[1] == whole
