"""Full-size parity: the CUDA path against stored oracle sets (tests/golden/).

Each golden file was written by tests/golden/make_golden.py from the CPU oracle alone; the
instance is regenerated here from the seed and sizes in the file's header.  Files with an
x range hold the set of the subproblems of those l-mers of S_1 (Section 2.3), and the
GPU solves the same range.  The (17,6) files are the instances bench.py times.
"""

from __future__ import annotations

import os

import pytest

from conftest import golden_module

pytestmark = pytest.mark.gpu

G = golden_module()
CASES = [name for name in G.CASES if os.path.exists(G.path(name))]


@pytest.mark.parametrize("name", CASES)
def test_golden_case(name):
    from paper_1307_0571_gb300 import build, pms
    build.build()
    meta, want = G.load(name)
    case = G.CASES[name]
    inst = G.instance(case)
    assert str(inst.seed) == meta["seed"]
    assert inst.motif == meta["planted"]
    xb, xe = (int(v) for v in meta["x_range"].split())
    with pms.Context(0, x_begin=xb, x_end=xe) as ctx:
        got = ctx.solve(inst.seqs, case["n"], case["m"], case["alphabet"], case["l"],
                        case["d"])
    assert len(got) == int(meta["count"])
    assert got == want


def test_golden_files_exist():
    assert len(CASES) >= 8
