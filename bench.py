#!/usr/bin/env python
"""Benchmark of the GB300 planted-motif-search path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one exact solve of one planted DNA (17,6) instance with n=20 strings of length
m=600 (the paper's benchmark family, Section 1): packing, the 2d filter, the stack search
with Theorem 1 filtering and Algorithm 1 enumeration, verification, sort and duplicate
removal, all in libpms's CUDA kernels.  Each step solves a different seeded instance.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and a device
synchronise; each step is timed with CUDA events on the stream it runs on, and a
256 MiB buffer is rewritten before every step (outside the events) so L2 starts cold.
With N > 1 (launched by torchrun) every rank solves its own instances (replicas; the
subproblems need no exchange), the slowest rank's time counts, and `value` is the
whole-job instances per second.

The JSON line also carries: `e2e` (the same metric through pms_solve with the strings in
pinned host memory, copies included), `roofline` (search kernel, algorithmic integer ops
per second against the issue-limited integer peak), `cpu_baseline` (the CPU oracle on a
bounded sample, rank 0, N = 1 only), `clocks` (nvidia-smi sampled during the timed
region) and `gpu_launches` (kernels of libpms launched in the timed region).

--impl reference times the CPU oracle (the reference arm of this repository) on bounded
samples of the same workload and prints the same line with "impl": "reference".

--mode batched solves the 64-instance mixed batch ((l,d) in {(13,4),(15,5),(17,6)}, n in
{10,20,30}, m in {300,600,1000}) as one pms_solve_batch call and as 64 pms_solve calls, and
reports both throughputs and the per-instance p50/p99 of the single solves.  --mode
serving replays a Poisson stream of planted requests ((l,d) in {(13,4),...,(19,7)}, n in
[10,30], m in [300,1200]) through pms_submit/pms_poll at 0.8x the one-at-a-time rate and
reports p50/p99 latency (arrival to result) and throughput against solving the same
requests one at a time.  Both check that every result equals the one-at-a-time solve.
"""

from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solve time per (l,d) instance; l-mer Hd compares/s vs roofline; batched p99"
UNIT = "instances/s"
# The timed workload (default dna_17_6); the others exist for profiling smaller and larger
# cases of the same kernels.
WORKLOADS = {
    "dna_17_6": (dict(l=17, d=6, n=20, m=600, alphabet="ACGT"), 2),
    "dna_13_4": (dict(l=13, d=4, n=20, m=600, alphabet="ACGT"), 1),
    "dna_15_5": (dict(l=15, d=5, n=20, m=600, alphabet="ACGT"), 2),
    "dna_19_7": (dict(l=19, d=7, n=20, m=600, alphabet="ACGT"), 2),
    "dna_21_8": (dict(l=21, d=8, n=20, m=600, alphabet="ACGT"), 2),
}
WORKLOAD, SEED_CONFIG = WORKLOADS["dna_17_6"]   # seeds synth.workload_seed(config, j)


def _workload_name(w):
    return (f"planted DNA (l,d)=({w['l']},{w['d']}), n={w['n']}, m={w['m']} "
            f"(one instance per step)")
# dram__bytes_read.sum + dram__bytes_write.sum of the first search pass of a (17,6)
# solve at threshold 4 (one ncu --set full capture of the current kernel)
SEARCH_TRAFFIC_17_6 = 21.204e9 + 16.017e9
SM_COUNT = 152
INT_OPS_PER_CLK_SM = 128         # 4 SMSPs x 32 lanes issue-limited integer ops
POPC_PER_CLK_SM = 16             # popcount throughput per SM per clock
HD_TEST_OPS = 4                  # one DNA Hd test: 2 plane logic ops, popcount, compare
CPU_SAMPLE_X = 24                # l-mers of S_1 in the CPU baseline sample
CPU_SAMPLE_X1 = 2                # l-mers of S_1 in its one-thread sample
REF_SAMPLE_X = 0                 # l-mers of S_1 per reference-arm step (0: one per core)


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _rank_info():
    return _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)


def _seed(rank: int, j: int) -> int:
    from paper_1307_0571_gb300 import synth
    return synth.workload_seed(SEED_CONFIG, 1000 * rank + j)


def _max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it ("model name", or the Arm part number)."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read().splitlines()
    except OSError:
        return platform.machine()
    fields = {}
    for ln in info:
        k, _, v = ln.partition(":")
        fields.setdefault(k.strip(), v.strip())
    if fields.get("model name"):
        return fields["model name"]
    if fields.get("CPU part"):
        return (f"{platform.machine()} CPU implementer {fields.get('CPU implementer', '?')} "
                f"part {fields['CPU part']}")
    return platform.machine()


def cpu_baseline(inst, l, d, n, m, sample_x=CPU_SAMPLE_X, sample_x1=CPU_SAMPLE_X1) -> dict:
    """The PMS8 oracle (plain CPU C, all host cores) on the subproblems of the first
    `sample_x` l-mers of S_1, scaled to whole instances per second; and the same on one
    thread for the first `sample_x1` l-mers."""
    import oracle
    oracle.build()
    L = m - l + 1
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.motifs_pms8(inst.seqs, n, m, "ACGT", l, d, t=3, x_begin=0, x_end=sample_x,
                       threads=cores)
    dt = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.motifs_pms8(inst.seqs, n, m, "ACGT", l, d, t=3, x_begin=0, x_end=sample_x1,
                       threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": (sample_x / L) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": _cpu_model(),
            "sample": f"PMS8 oracle (oracle/pms_oracle.c, threshold 3) on the subproblems of "
                      f"l-mers 0..{sample_x - 1} of S_1 ({sample_x}/{L} of one instance) "
                      f"took {dt:.2f} s; value scales that to whole instances",
            "one_thread": {"value": (sample_x1 / L) / dt1, "unit": UNIT, "cores": 1,
                           "sample": f"l-mers 0..{sample_x1 - 1} of S_1 on one thread took "
                                     f"{dt1:.2f} s"}}


def run_reference(args) -> None:
    rank, world, _ = _rank_info()
    if rank != 0:
        return
    import oracle
    from paper_1307_0571_gb300 import synth
    oracle.build()
    W_ = WORKLOAD
    L = W_["m"] - W_["l"] + 1
    cores = os.cpu_count() or 1
    per_step = min(REF_SAMPLE_X or cores, L)
    times, xs = [], 0
    for j in range(args.warmup + args.steps):
        inst = synth.planted_instance(_seed(0, j), W_["n"], W_["m"], W_["l"], W_["d"])
        t0 = time.perf_counter()
        oracle.motifs_pms8(inst.seqs, W_["n"], W_["m"], "ACGT", W_["l"], W_["d"], t=3,
                           x_begin=0, x_end=per_step, threads=cores)
        dt = time.perf_counter() - t0
        if j >= args.warmup:
            times.append(dt)
            xs += per_step
    total = sum(times)
    value = (xs / L) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": _workload_name(WORKLOAD), "sample": f"{per_step} l-mers of S_1 per step",
                   "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu_model": _cpu_model(),
                         "sample": f"each step: PMS8 oracle on the subproblems of l-mers "
                                   f"0..{per_step - 1} of S_1 of a fresh instance"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args) -> None:
    import torch
    rank, world, local = _rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1307_0571_gb300 import pms, synth
    W_ = WORKLOAD
    l, d, n, m = W_["l"], W_["d"], W_["n"], W_["m"]
    ctx = pms.Context(local, threshold=args.threshold)
    total_steps = args.warmup + args.steps
    insts = [synth.planted_instance(_seed(rank, j), n, m, l, d) for j in range(total_steps)]
    dseqs = [torch.frombuffer(bytearray(i.seqs), dtype=torch.uint8).to("cuda") for i in insts]
    cap = 1 << 16
    dout = torch.empty(cap * l, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]

    def step(j):
        return ctx.solve_device(dseqs[j].data_ptr(), n, m, "ACGT", l, d, dout.data_ptr(), cap,
                                stream.cuda_stream)

    for j in range(args.warmup):
        flush.fill_(j & 0xFF)
        step(j)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    _barrier(world)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    stats, counts = [], []
    for i in range(args.steps):
        j = args.warmup + i
        flush.fill_(j & 0xFF)
        ev[i][0].record(stream)
        cnt, st = step(j)
        ev[i][1].record(stream)
        stats.append(st)
        counts.append(cnt)
    torch.cuda.synchronize()
    _barrier(world)
    t_wall1 = time.perf_counter()
    clocks = sampler.stop()

    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = _max_over_ranks(sum(step_ms), world)
    value = world * args.steps / (total_ms / 1000.0)
    search_ms = [st.search_ms for st in stats]
    ops = [st.search_ops for st in stats]
    launches = sum(st.launches for st in stats)
    compares = sum(st.hd_compares for st in stats)
    achieved_ops = sum(ops) / (sum(search_ms) / 1000.0)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak_ops = SM_COUNT * INT_OPS_PER_CLK_SM * sm_max * 1e6
    peak_popc = SM_COUNT * POPC_PER_CLK_SM * sm_max * 1e6

    # end to end: pms_solve with the strings in pinned host memory, result read back
    pinned = [torch.frombuffer(bytearray(i.seqs), dtype=torch.uint8).pin_memory()
              for i in insts]
    for j in range(args.warmup):
        ctx.solve_ptr(pinned[j].data_ptr(), n, m, "ACGT", l, d)
    _barrier(world)
    t0 = time.perf_counter()
    e2e_stats = []
    found_planted = 0
    for i in range(args.steps):
        j = args.warmup + i
        res = ctx.solve_ptr(pinned[j].data_ptr(), n, m, "ACGT", l, d)
        e2e_stats.append(ctx.last_stats)
        found_planted += insts[j].motif in res
    e2e_s = _max_over_ranks(time.perf_counter() - t0, world)
    if found_planted != args.steps:
        raise SystemExit(f"planted motif missing in {args.steps - found_planted} solves")

    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": _workload_name(WORKLOAD), "instances_per_rank": args.steps,
                   "threshold": stats[0].threshold, "parallelism": f"replicas x{world}",
                   "l2": "256 MiB buffer rewritten before every step (outside the events)",
                   "inputs": "strings resident in HBM; result left in HBM"},
        "solve_ms": {"mean": statistics.mean(step_ms), "p50": statistics.median(step_ms),
                     "max": max(step_ms)},
        "wall_ms_per_step": 1000 * (t_wall1 - t_wall0) / args.steps,
        "hd_compares_per_s": compares / (sum(search_ms) / 1000.0),
        # Hd/Cd tests of the search against the compares peak: the smaller of the integer
        # issue peak over the ops of one DNA Hd test (2 plane XORs/ORs, popcount, compare)
        # and the popcount peak over its one popcount
        "hd_compares": {
            "per_s": compares / (sum(search_ms) / 1000.0),
            "peak_per_s": min(peak_ops / HD_TEST_OPS, peak_popc),
            "frac": (compares / (sum(search_ms) / 1000.0)) / min(peak_ops / HD_TEST_OPS, peak_popc),
            "peak_note": f"min({SM_COUNT} SMs x {INT_OPS_PER_CLK_SM} int ops/clk / "
                         f"{HD_TEST_OPS} ops per test, {SM_COUNT} SMs x {POPC_PER_CLK_SM} "
                         f"popc/clk) x {sm_max:.0f} MHz"},
        "roofline": {"kernel": "search_kernel", "bound": "alu",
                     "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tintop/s", "frac": achieved_ops / peak_ops,
                     # DRAM bytes of the first search pass of a (17,6) solve (ncu capture
                     # in profiles/search_kernel_dna_17_6.md); other workloads: not captured
                     "traffic": (SEARCH_TRAFFIC_17_6 if WORKLOAD is WORKLOADS["dna_17_6"][0]
                                 and stats[0].threshold == 4 else None),
                     "peak_note": f"{SM_COUNT} SMs x {INT_OPS_PER_CLK_SM} int ops/clk x "
                                  f"{sm_max:.0f} MHz (derived; no measured integer peak)"},
        "e2e": {"value": world * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": statistics.mean(s.h2d_bytes for s in e2e_stats),
                "d2h_bytes_per_step": statistics.mean(s.d2h_bytes for s in e2e_stats)},
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(insts[0], l, d, n, m)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))]


def run_batched(args) -> None:
    from paper_1307_0571_gb300 import pms, synth
    insts = synth.batched_mix(synth.workload_seed(3, 0), 64)
    P = [pms.Instance(i.seqs, i.n, i.m, "ACGT", i.l, i.d) for i in insts]
    ctx = pms.Context(0)
    singles = [ctx.solve(p.seqs, p.n, p.m, "ACGT", p.l, p.d) for p in P]   # warm-up, tuning
    seq_s, lat = [], []
    batch_s = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        for p in P:
            t1 = time.perf_counter()
            ctx.solve(p.seqs, p.n, p.m, "ACGT", p.l, p.d)
            lat.append(time.perf_counter() - t1)
        seq_s.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        got = ctx.solve_batch(P)
        batch_s.append(time.perf_counter() - t0)
        if got != singles:
            raise SystemExit("batched result differs from single solves")
    seq, bat = statistics.median(seq_s), statistics.median(batch_s)
    print(json.dumps({
        "mode": "batched", "metric": METRIC, "value": len(P) / bat, "unit": UNIT,
        "n_gpus": 1, "steps": len(batch_s), "higher_is_better": True, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "64 planted DNA instances, (l,d) in {(13,4),(15,5),(17,6)}, "
                               "n in {10,20,30}, m in {300,600,1000}",
                   "motifs": sum(len(x) for x in singles)},
        "batched_s": bat, "sequential_s": seq,
        "sequential_instances_per_s": len(P) / seq, "speedup": seq / bat,
        "single_solve_ms": {"p50": 1000 * _pct(lat, 0.5), "p99": 1000 * _pct(lat, 0.99)},
        "identical_output": True}), flush=True)


def run_serving(args) -> None:
    from paper_1307_0571_gb300 import pms, synth
    nreq = args.requests
    proto = synth.serving_stream(synth.workload_seed(5, 0), nreq, rate_per_s=1.0)
    insts = [inst for _, inst in proto]
    ctx = pms.Context(0)
    # one at a time (also warms up and tunes every class)
    alone, t_alone = [], []
    for inst in insts:
        t0 = time.perf_counter()
        alone.append(ctx.solve(inst.seqs, inst.n, inst.m, "ACGT", inst.l, inst.d))
        t_alone.append(time.perf_counter() - t0)
    seq_rate = len(insts) / sum(t_alone)
    rate = 0.8 * seq_rate if args.rate < 0 else args.rate
    if rate > 0:
        stream = synth.serving_stream(synth.workload_seed(5, 0), nreq, rate_per_s=rate)
    else:   # saturation: every request arrives at time 0
        stream = [(0.0, inst) for inst in insts]
    t0 = time.perf_counter()
    tickets, arrivals = [], []
    pending = {}
    done = {}
    i = 0
    while len(done) < len(stream):
        now = time.perf_counter() - t0
        while i < len(stream) and stream[i][0] <= now:
            a, inst = stream[i]
            tk = ctx.submit(pms.Instance(inst.seqs, inst.n, inst.m, "ACGT", inst.l, inst.d))
            pending[tk] = (i, a)
            i += 1
        for tk in list(pending):
            r = ctx.poll(tk)
            if r is not None:
                j, a = pending.pop(tk)
                done[j] = (r, time.perf_counter() - t0 - a)
        time.sleep(0.0005)
    total = time.perf_counter() - t0
    if any(done[j][0] != alone[j] for j in range(len(stream))):
        raise SystemExit("served result differs from the solve alone")
    lat = [done[j][1] for j in range(len(stream))]
    print(json.dumps({
        "mode": "serving", "metric": METRIC, "value": len(stream) / total, "unit": UNIT,
        "n_gpus": 1, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"{nreq} planted DNA requests, (l,d) in {{(13,4),(15,5),"
                               "(17,6),(19,7)}, n in [10,30], m in [300,1200], Poisson",
                   "arrival_rate_per_s": rate if rate > 0 else "all at t=0", "slots": 2},
        "latency_ms": {"p50": 1000 * _pct(lat, 0.5), "p99": 1000 * _pct(lat, 0.99),
                       "max": 1000 * max(lat)},
        "one_at_a_time_instances_per_s": seq_rate,
        "one_at_a_time_latency_ms": {"p50": 1000 * _pct(t_alone, 0.5),
                                     "p99": 1000 * _pct(t_alone, 0.99)},
        "identical_output": True}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="dna_17_6")
    ap.add_argument("--threshold", type=int, default=0, help="0 = autotuned")
    ap.add_argument("--mode", choices=["single", "batched", "serving"], default="single")
    ap.add_argument("--requests", type=int, default=120, help="serving mode: requests")
    ap.add_argument("--rate", type=float, default=-1.0,
                    help="serving mode: arrivals/s (-1: 0.8x one-at-a-time, 0: all at once)")
    args = ap.parse_args()
    global WORKLOAD, SEED_CONFIG
    WORKLOAD, SEED_CONFIG = WORKLOADS[args.workload]
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
