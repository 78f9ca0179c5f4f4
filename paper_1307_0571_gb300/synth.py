"""Seeded synthetic planted-motif instances (the paper's benchmark family, Section 1).

The paper evaluates only on synthetic inputs: n i.i.d. uniform strings of length m over
an alphabet, with one random l-mer planted at a random position of every string and each
planted copy changed in d positions (the recipe of Section 1, which Section 3 uses for
every measurement).  This module is the one
place that draws those inputs; it holds none of the motif-search arithmetic, so both the
CUDA path and the CPU oracle can be fed from it.

Random numbers
--------------
Every draw is the i-th output of a SplitMix64 sequence (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): with gamma = 0x9E3779B97F4A7C15,
output i of the sequence keyed by k is mix64(k + (i + 1) * gamma), where mix64 is the
published SplitMix64 finaliser.  The generator is counter based, so it vectorises in numpy
and gives the same bytes on every machine.  The key of stream s under seed S is
mix64(S * gamma ^ (s + 1) * 0xD1B54A32D192ED03).  A draw x maps to a uniform integer below k
by ((x >> 32) * k) >> 32 (bias below k / 2**32).

Draw order of one instance (seed S, alphabet of size k, n strings, length m, planted l-mer
with exactly d changes per copy):
  stream 0, draws 0..l-1          -> the planted motif;
  stream 1+i, draws 0..m-1        -> background of string i;
  stream 1+i, draw m              -> plant position, uniform in [0, m-l];
  stream 1+i, draws m+1..m+d      -> partial Fisher-Yates over [0, l): the d changed positions;
  stream 1+i, draws m+1+d..m+2d   -> replacement letters, uniform over the k-1 other letters.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
STREAM_MUL = 0xD1B54A32D192ED03
MASK64 = (1 << 64) - 1

DNA = "ACGT"
PROTEIN = "ACDEFGHIKLMNPQRSTVWY"


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= np.uint64(0xBF58476D1CE4E5B9)
    z ^= z >> np.uint64(27)
    z *= np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> int:
    k = ((seed * GAMMA) & MASK64) ^ (((stream + 1) * STREAM_MUL) & MASK64)
    return int(_mix64(np.array([k], dtype=np.uint64))[0])


def draws(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Draws start..start+count-1 of stream `stream` under `seed`, as uint64."""
    key = np.uint64(stream_key(seed, stream))
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + idx * np.uint64(GAMMA))


def uniform_below(x: np.ndarray, k) -> np.ndarray:
    """Map uint64 draws to integers in [0, k) (k may be an array)."""
    return ((x >> np.uint64(32)) * np.asarray(k, dtype=np.uint64)) >> np.uint64(32)


@dataclass
class Instance:
    """One planted (l, d) instance: n strings of length m over `alphabet`."""

    seqs: bytes                     # n*m bytes, row-major, letters of `alphabet`
    n: int
    m: int
    alphabet: str
    l: int
    d: int
    motif: str = ""                 # the planted l-mer
    positions: list = field(default_factory=list)  # plant position per string
    seed: int = 0

    def rows(self) -> list[str]:
        s = self.seqs.decode("ascii")
        return [s[i * self.m:(i + 1) * self.m] for i in range(self.n)]


def planted_instance(seed: int, n: int, m: int, l: int, d: int,
                     alphabet: str = DNA) -> Instance:
    """Generate the planted instance described in the module docstring."""
    k = len(alphabet)
    if not (1 <= l <= m and 0 <= d <= l and k >= 2):
        raise ValueError("need 1 <= l <= m, 0 <= d <= l and an alphabet of >= 2 letters")
    letters = np.frombuffer(alphabet.encode("ascii"), dtype=np.uint8)
    motif = uniform_below(draws(seed, 0, 0, l), k).astype(np.int64)
    out = np.empty((n, m), dtype=np.int64)
    positions = []
    for i in range(n):
        r = draws(seed, 1 + i, 0, m + 1 + 2 * d)
        row = uniform_below(r[:m], k).astype(np.int64)
        pos = int(uniform_below(r[m:m + 1], m - l + 1)[0])
        perm = list(range(l))
        for t in range(d):
            j = t + int(uniform_below(r[m + 1 + t:m + 2 + t], l - t)[0])
            perm[t], perm[j] = perm[j], perm[t]
        copy = motif.copy()
        for t in range(d):
            c = perm[t]
            u = int(uniform_below(r[m + 1 + d + t:m + 2 + d + t], k - 1)[0])
            copy[c] = (copy[c] + 1 + u) % k
        row[pos:pos + l] = copy
        out[i] = row
        positions.append(pos)
    seqs = letters[out].tobytes()
    return Instance(seqs=seqs, n=n, m=m, alphabet=alphabet, l=l, d=d,
                    motif=letters[motif].tobytes().decode("ascii"),
                    positions=positions, seed=seed)


def random_instance(seed: int, n: int, m: int, l: int, d: int,
                    alphabet: str = DNA) -> Instance:
    """i.i.d. uniform strings with nothing planted (stream 1+i, draws 0..m-1)."""
    k = len(alphabet)
    letters = np.frombuffer(alphabet.encode("ascii"), dtype=np.uint8)
    out = np.stack([uniform_below(draws(seed, 1 + i, 0, m), k).astype(np.int64)
                    for i in range(n)])
    return Instance(seqs=letters[out].tobytes(), n=n, m=m, alphabet=alphabet, l=l, d=d,
                    seed=seed)


# Seeds of the standard workloads: instance j of workload c uses SEED_BASE + 100*c + j.
SEED_BASE = 0x504D5338 * 1000


def workload_seed(config: int, j: int) -> int:
    return SEED_BASE + 100 * config + j


def batched_mix(seed: int, count: int = 64):
    """The mixed batch: (l,d) from {(13,4),(15,5),(17,6)}, n from {10,20,30},
    m from {300,600,1000}, one planted DNA instance per draw (stream 0x100 picks the
    parameters, instance j uses seed*1000 + j)."""
    r = draws(seed, 0x100, 0, 3 * count)
    ld = [(13, 4), (15, 5), (17, 6)]
    ns = [10, 20, 30]
    ms = [300, 600, 1000]
    out = []
    for j in range(count):
        a, b, c = (int(v) for v in uniform_below(r[3 * j:3 * j + 3], 3))
        l, d = ld[a]
        out.append(planted_instance(seed * 1000 + j, ns[b], ms[c], l, d))
    return out


def serving_stream(seed: int, count: int = 2000, rate_per_s: float = 100.0):
    """Serving requests: (l,d) uniform over {(13,4),(15,5),(17,6),(19,7)}, n uniform in
    [10,30], m uniform in [300,1200], Poisson arrivals at `rate_per_s` (exponential gaps
    from stream 0x200).  Returns [(arrival_s, Instance)]."""
    r = draws(seed, 0x200, 0, 4 * count)
    ld = [(13, 4), (15, 5), (17, 6), (19, 7)]
    t = 0.0
    out = []
    for j in range(count):
        a = int(uniform_below(r[4 * j:4 * j + 1], 4)[0])
        n = 10 + int(uniform_below(r[4 * j + 1:4 * j + 2], 21)[0])
        m = 300 + int(uniform_below(r[4 * j + 2:4 * j + 3], 901)[0])
        u = (int(r[4 * j + 3]) >> 11) * (1.0 / (1 << 53))
        t += -np.log1p(-u) / rate_per_s
        l, d = ld[a]
        out.append((t, planted_instance(seed * 10000 + j, n, m, l, d)))
    return out
