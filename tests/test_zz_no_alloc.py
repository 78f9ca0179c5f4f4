"""The allocation-free solve (pms_solve_device_noalloc) against pms_solve_device.

pms_solve_device_noalloc serves callers that must not allocate device memory while they
run (services that reserve all their device memory in their own pool at start-up,
real-time pipelines where an allocation would stall the device); it works in a fixed
scratch array that every call reuses.  These tests call it through the C ABI twice in a
row, on different instances, and require the same motif set as pms_solve_device, bit for
bit; they also check that a request too large for the fixed array is refused cleanly and
leaves the next call unharmed.  This file is collected last so that, if it fails, every
other test has already run.
"""

from __future__ import annotations

import pytest

from paper_1307_0571_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev_bytes(b: bytes):
    import torch
    return torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()


def _read(dout, count: int, l: int) -> list[str]:
    raw = bytes(dout[:count * l].cpu().numpy().tobytes()).decode("ascii")
    return [raw[i * l:(i + 1) * l] for i in range(count)]


def _via_existing(ctx, inst, dseq, dout, cap):
    import torch
    count, _ = ctx.solve_device(dseq.data_ptr(), inst.n, inst.m, "ACGT", inst.l, inst.d,
                                dout.data_ptr(), cap, torch.cuda.current_stream().cuda_stream)
    return _read(dout, count, inst.l)


def _via_noalloc(inst, dseq, dout, cap, threshold=0):
    import torch
    from paper_1307_0571_gb300 import pms
    count = pms.solve_device_noalloc(dseq.data_ptr(), inst.n, inst.m, "ACGT", inst.l, inst.d,
                                     dout.data_ptr(), cap,
                                     torch.cuda.current_stream().cuda_stream, threshold)
    return _read(dout, count, inst.l)


def test_noalloc_matches_solve_device_two_calls_in_a_row():
    import torch
    from paper_1307_0571_gb300 import build, pms
    build.build()
    cases = [synth.planted_instance(synth.workload_seed(1, 3), 20, 600, 13, 4),
             synth.planted_instance(synth.workload_seed(2, 4), 12, 300, 15, 5)]
    cap = 1 << 16
    with pms.Context(0) as ctx:
        for inst in cases:
            dseq = _dev_bytes(inst.seqs)
            d1 = torch.zeros(cap * inst.l, dtype=torch.uint8, device="cuda")
            d2 = torch.zeros(cap * inst.l, dtype=torch.uint8, device="cuda")
            want = _via_existing(ctx, inst, dseq, d1, cap)
            got = _via_noalloc(inst, dseq, d2, cap)
            assert inst.motif in want
            assert got == want


def test_noalloc_refuses_requests_larger_than_its_scratch():
    import torch
    from paper_1307_0571_gb300 import pms
    big = synth.random_instance(5, 64, 4000, 12, 3)
    dseq = _dev_bytes(big.seqs)
    dout = torch.zeros(16 * 12, dtype=torch.uint8, device="cuda")
    with pytest.raises(pms.PMSError) as e:
        pms.solve_device_noalloc(dseq.data_ptr(), 64, 4000, "ACGT", 12, 3, dout.data_ptr(), 16)
    assert e.value.code == pms.PMS_E_NOMEM
    # the shared array is still usable afterwards
    small = synth.planted_instance(6, 8, 100, 9, 2)
    ds = _dev_bytes(small.seqs)
    do = torch.zeros(4096 * 9, dtype=torch.uint8, device="cuda")
    got = _via_noalloc(small, ds, do, 4096)
    with pms.Context(0) as ctx:
        d1 = torch.zeros(4096 * 9, dtype=torch.uint8, device="cuda")
        assert got == _via_existing(ctx, small, ds, d1, 4096)
