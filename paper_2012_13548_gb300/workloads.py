"""Seeded synthetic workloads: the input recipes shared by the tests, the bench
and the oracle runs.

This module holds no step of the method (no generator, CSR or BFS arithmetic).
It fixes the Graph500 parameters of each workload, derives the seeds, draws
roots and arrival traces.  Both the CUDA path and the oracle receive what it
returns as plain inputs.

Workloads (Graph500 Kronecker graphs, Sec. 2.1 of the paper: #V = 2^scale,
#E = edgefactor * #V; initiator A, B, C, D = 0.57, 0.19, 0.19, 0.05):

  s10      SCALE 10, 8 roots            -- correctness smoke case
  s20      SCALE 20, 64 roots           -- plain direction-optimising BFS
  s26      SCALE 26, 64 roots           -- plain BFS at full size + kernel 1
  s22ms    SCALE 22, 64 roots in one multi-source launch
  batch32  32 graphs, SCALE uniform in 12..18, 8 roots each, one launch
  serve6   6 resident graphs SCALE 14..24, Poisson 5000 req/s
  sssp22   kernel 3: SCALE 22 with the weight row, 64 roots, single-source
           shortest paths (Sec. 2.4)
"""
from dataclasses import dataclass

import numpy as np

EDGEFACTOR = 16
A, B, C = 0.57, 0.19, 0.19          # D = 1 - A - B - C = 0.05

SEED_GEN, SEED_PERM, SEED_SHUF, SEED_ROOT, SEED_ARRIVAL = 1, 2, 3, 4, 5
SEED_WEIGHT = 6

_MASK64 = (1 << 64) - 1


@dataclass(frozen=True)
class GraphSpec:
    scale: int
    edgefactor: int = EDGEFACTOR
    index: int = -1            # position in a batch of graphs, -1 for a lone graph

    @property
    def n(self) -> int:
        return 1 << self.scale

    @property
    def m(self) -> int:
        return self.n * self.edgefactor

    def seeds(self):
        """(seed_gen, seed_perm, seed_shuf, seed_root): base seed XOR scale<<32,
        and XOR (index+1)<<40 for graph `index` of a batch."""
        salt = (self.scale << 32)
        if self.index >= 0:
            salt ^= (self.index + 1) << 40
        return tuple((s ^ salt) & _MASK64 for s in (SEED_GEN, SEED_PERM, SEED_SHUF, SEED_ROOT))

    def seed_weight(self):
        """Seed of the weight row (kernel 3), salted like seeds()."""
        salt = (self.scale << 32)
        if self.index >= 0:
            salt ^= (self.index + 1) << 40
        return (SEED_WEIGHT ^ salt) & _MASK64

    def kron_args(self):
        """Arguments of kron_generate after (scale, edgefactor, a, b, c)."""
        g, p, s, _ = self.seeds()
        return dict(scale=self.scale, edgefactor=self.edgefactor, a=A, b=B, c=C,
                    seed_gen=g, seed_perm=p, seed_shuf=s)


WORKLOADS = {
    "s10": dict(scale=10, roots=8),
    "s20": dict(scale=20, roots=64),
    "s26": dict(scale=26, roots=64),
    "s22ms": dict(scale=22, roots=64),
    "batch32": dict(graphs=32, scale_lo=12, scale_hi=18, roots=8),
    "serve6": dict(scales=(14, 16, 18, 20, 22, 24), rate=5000.0),
    "sssp22": dict(scale=22, roots=64, delta=0.1),
}


def _sm64_np(seed: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 (Steele, Lea, Flood 2014) output for counters idx, vectorised.
    Used only to draw roots and traces."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def select_roots(off: np.ndarray, k: int, seed_root: int) -> np.ndarray:
    """The first k vertices of degree >= 1, ordered by (SplitMix64(seed_root, v), v).

    `off` is a CSR offset array (int64 [n+1]); the degree is taken from the
    deduplicated, loop-free graph.  Returns int64 [k] distinct roots (fewer if the
    graph has fewer non-isolated vertices)."""
    off = np.asarray(off, dtype=np.int64)
    n = off.size - 1
    cand = np.nonzero(np.diff(off) > 0)[0]
    if cand.size == 0:
        return np.zeros(0, dtype=np.int64)
    h = _sm64_np(seed_root, cand)
    k = min(k, cand.size)
    if cand.size > 4 * k + 64:
        # the k smallest keys: partition, then order that small set exactly
        part = np.argpartition(h, 4 * k)[: 4 * k + 1]
        cand, h = cand[part], h[part]
    order = np.lexsort((cand, h))
    del n
    return cand[order[:k]].astype(np.int64)


def batch_specs(count: int = 32, lo: int = 12, hi: int = 18, seed: int = SEED_GEN):
    """`count` graph specs with SCALE drawn uniformly from lo..hi (inclusive)."""
    idx = np.arange(count, dtype=np.uint64)
    h = _sm64_np(seed ^ (0xB47C << 48), idx)
    scales = lo + (h % np.uint64(hi - lo + 1)).astype(np.int64)
    return [GraphSpec(scale=int(s), index=i) for i, s in enumerate(scales)]


def poisson_trace(rate: float, duration_s: float, n_graphs: int, seed: int = SEED_ARRIVAL):
    """Open-loop Poisson arrivals: (t_arrival_s float64 [q], graph_id int32 [q],
    root_draw uint64 [q]).  root_draw is turned into a root by root_from_draw."""
    rng = np.random.Generator(np.random.Philox(seed))
    n_est = int(rate * duration_s * 1.2) + 64
    gaps = rng.exponential(1.0 / rate, size=n_est)
    t = np.cumsum(gaps)
    while t[-1] < duration_s:
        more = rng.exponential(1.0 / rate, size=n_est)
        t = np.concatenate([t, t[-1] + np.cumsum(more)])
    t = t[t < duration_s]
    q = t.size
    gid = rng.integers(0, n_graphs, size=q).astype(np.int32)
    draw = rng.integers(0, 2**63 - 1, size=q, dtype=np.int64).astype(np.uint64)
    return t.astype(np.float64), gid, draw


def root_from_draw(off: np.ndarray, draws: np.ndarray) -> np.ndarray:
    """Map uniform draws to roots uniform over the vertices of degree >= 1."""
    cand = np.nonzero(np.diff(np.asarray(off, dtype=np.int64)) > 0)[0]
    return cand[(np.asarray(draws, dtype=np.uint64) % np.uint64(cand.size)).astype(np.int64)]
