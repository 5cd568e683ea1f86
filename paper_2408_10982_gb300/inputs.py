"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only makes inputs: R-MAT graphs in in-CSR form, quantised edge
probabilities and query/arrival parameters.  It holds none of the method's
arithmetic (no RRR sampling, no coverage, no greedy): the random numbers the
method itself draws (roots, coins, partition labels) are produced on each side
by its own Philox4x32-10.

Graph layout (the paper replicates the whole graph on every machine and
samples over in-edges, Sec. 3.2 / S1):
  in_off  int64[n+1]  in-CSR offsets, edges sorted by (dst, src)
  in_src  int32[m]    source vertex of each in-edge; edge id e = CSR position
  w       uint32[m]   edge probability quantised to 32 bits: an IC edge is live
                      when a uniform 32-bit draw is below w[e]; for LT, w[e] is
                      the probability that dst picks this in-edge.

The paper's inputs are SNAP/KONECT social networks (Table 3).  They are not
available here, so R-MAT graphs with the same vertex/edge counts stand in for
them.  R-MAT candidates come from a splitmix64 stream (C, inputs_rmat.c);
per-edge weight draws from numpy's PCG64 raw output (stable across numpy
versions); both are keyed by the given seed.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

TWO32 = 1 << 32
U32_MAX = TWO32 - 1
RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19


@dataclass
class Graph:
    """A directed graph in in-CSR form (see the module docstring)."""
    n: int
    in_off: np.ndarray
    in_src: np.ndarray
    w: np.ndarray

    @property
    def m(self) -> int:
        return int(self.in_src.shape[0])

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (self.in_off, self.in_src, self.w):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()[:16]


def _u32_stream(bitgen: np.random.PCG64, count: int) -> np.ndarray:
    raw = bitgen.random_raw((count + 1) // 2)
    return raw.view(np.uint32)[:count]


def quantise_probability(p: float) -> int:
    """Round a probability to the uint32 threshold used by the coin test."""
    return min(int(math.floor(p * TWO32 + 0.5)), U32_MAX)


_RMAT_LIB = None


def _rmat_lib():
    """Load (compiling on first use) the C R-MAT fixture next to this file."""
    global _RMAT_LIB
    if _RMAT_LIB is None:
        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "inputs_rmat.c")
        so = os.path.join(here, "_inputs_rmat.so")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = f"{so}.{os.getpid()}.tmp"
            subprocess.run(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-pthread", src, "-o", tmp],
                           check=True)
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        lib.rmat_generate.restype = ctypes.c_int64
        lib.rmat_generate.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
        _RMAT_LIB = lib
    return _RMAT_LIB


def rmat_edges(n: int, m: int, seed: int = 42, levels: int | None = None,
               a: float = RMAT_A, b: float = RMAT_B,
               c: float = RMAT_C) -> tuple[np.ndarray, np.ndarray]:
    """Directed R-MAT edge list (src -> dst means src influences dst).

    Candidates are drawn in order; each picks one of four quadrants per level
    by comparing a 32-bit draw with the cumulative a, a+b, a+b+c thresholds
    (quadrant a = (0,0), b = (0,1), c = (1,0), d = (1,1) for (src bit, dst
    bit)).  Candidates with an endpoint >= n, self-loops and repeats of an
    earlier candidate are dropped; generation stops once exactly m distinct
    edges have been accepted.  The stream and the dedup run in C
    (inputs_rmat.c).
    """
    if levels is None:
        levels = max(1, int(math.ceil(math.log2(max(n, 2)))))
    if n < 2 or m > n * (n - 1) // 2:
        raise ValueError("R-MAT request too dense for a simple digraph")
    t1 = int(math.floor(a * TWO32))
    t2 = int(math.floor((a + b) * TWO32))
    t3 = int(math.floor((a + b + c) * TWO32))
    src = np.empty(m, dtype=np.int64)
    dst = np.empty(m, dtype=np.int64)
    got = _rmat_lib().rmat_generate(n, m, levels, seed & (TWO32 * TWO32 - 1), t1, t2, t3,
                                    src.ctypes.data, dst.ctypes.data)
    if got != m:
        raise RuntimeError(f"R-MAT generator accepted {got} of {m} edges")
    return src, dst


def in_csr(n: int, src: np.ndarray, dst: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Build in-CSR (edges sorted by (dst, src)) from a repeat-free edge list."""
    key = np.sort(dst.astype(np.int64) * n + src.astype(np.int64))
    in_src = (key % n).astype(np.int32)
    indeg = np.bincount(key // n, minlength=n).astype(np.int64)
    in_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(indeg, out=in_off[1:])
    return in_off, in_src


def weights_uniform(m: int, p: float) -> np.ndarray:
    """IC weights: the same probability p on every edge."""
    return np.full(m, quantise_probability(p), dtype=np.uint32)


def weights_trivalency(m: int, seed: int = 42,
                       values: tuple[float, ...] = (0.1, 0.01, 0.001)) -> np.ndarray:
    """IC weights drawn uniformly from a small set of probabilities, by edge id."""
    bg = np.random.PCG64(seed ^ 0x7472697661)
    r = _u32_stream(bg, m).astype(np.uint64)
    idx = (r * np.uint64(len(values))) >> np.uint64(32)
    table = np.array([quantise_probability(v) for v in values], dtype=np.uint32)
    return table[idx.astype(np.int64)]


def weights_inverse_indegree(in_off: np.ndarray) -> np.ndarray:
    """LT weights w(u,v) = 1/indeg(v), quantised so a vertex's weights sum to <= 2^32."""
    d = np.diff(in_off)
    per_v = np.where(d > 0, np.minimum(TWO32 // np.maximum(d, 1), U32_MAX), 0)
    return np.repeat(per_v.astype(np.uint32), d)


def _uniform_probabilities(m: int, seed: int, hi: float) -> np.ndarray:
    bg = np.random.PCG64(seed ^ 0x756e69)
    return _u32_stream(bg, m).astype(np.float64) / TWO32 * hi


def weights_uniform_random(m: int, seed: int, hi: float = 0.1) -> np.ndarray:
    """IC weights drawn U[0, hi] per edge (the paper's own weight model, Sec. 4.1)."""
    r = _uniform_probabilities(m, seed, hi)
    return np.minimum(np.floor(r * TWO32 + 0.5), U32_MAX).astype(np.uint32)


def weights_uniform_random_lt(in_off: np.ndarray, seed: int, hi: float = 0.1) -> np.ndarray:
    """LT weights from the same U[0, hi] draws: a vertex whose in-weights sum
    above 1 has them scaled to sum to 1 (the LT model needs sum <= 1), the
    others keep them; quantised down so every vertex's sum stays <= 2^32."""
    m = int(in_off[-1])
    r = _uniform_probabilities(m, seed, hi)
    d = np.diff(in_off)
    owner = np.repeat(np.arange(d.size), d)
    tot = np.bincount(owner, weights=r, minlength=d.size)
    scale = 1.0 / np.maximum(tot, 1.0)
    return np.minimum(np.floor(r * scale[owner] * TWO32), U32_MAX).astype(np.uint32)


def rmat_graph(n: int, m: int, seed: int = 42, weights: str = "ic0.1",
               levels: int | None = None) -> Graph:
    """R-MAT graph with one of the weight models used by the workloads.

    weights: "ic<p>" (uniform p), "trivalency", "lt" (1/in-degree),
    "u0.1" (IC, U[0, 0.1] per edge), "lt-u0.1" (LT from the same draws, each
    vertex's in-weights scaled to sum to at most 1).
    """
    src, dst = rmat_edges(n, m, seed=seed, levels=levels)
    in_off, in_src = in_csr(n, src, dst)
    if weights.startswith("ic"):
        w = weights_uniform(m, float(weights[2:]))
    elif weights == "trivalency":
        w = weights_trivalency(m, seed)
    elif weights == "lt":
        w = weights_inverse_indegree(in_off)
    elif weights.startswith("lt-u"):
        w = weights_uniform_random_lt(in_off, seed, float(weights[4:]))
    elif weights.startswith("u"):
        w = weights_uniform_random(m, seed, float(weights[1:]))
    else:
        raise ValueError(weights)
    return Graph(n, in_off, in_src, w)


def random_graph(n: int, m: int, seed: int, wmode: str = "random") -> Graph:
    """Small uniform random digraph (no self-loops, no repeats) for tests.

    wmode: "random" (uniform 32-bit weights), "lt" (1/in-degree), "zero",
    "one" (2^32-1), or a float string giving a uniform probability.
    """
    rng = np.random.default_rng(seed)
    pairs = [(u, v) for u in range(n) for v in range(n) if u != v]
    m = min(m, len(pairs))
    pick = rng.choice(len(pairs), size=m, replace=False)
    src = np.array([pairs[i][0] for i in pick], dtype=np.int64)
    dst = np.array([pairs[i][1] for i in pick], dtype=np.int64)
    in_off, in_src = in_csr(n, src, dst)
    if wmode == "random":
        w = rng.integers(0, TWO32, size=m, dtype=np.uint64).astype(np.uint32)
    elif wmode == "lt":
        w = weights_inverse_indegree(in_off)
    elif wmode == "lt_random":
        # random LT weights with per-vertex sum <= 2^32
        w = np.zeros(m, dtype=np.uint32)
        for v in range(n):
            b, e = int(in_off[v]), int(in_off[v + 1])
            if e > b:
                parts = rng.dirichlet(np.ones(e - b + 1))[: e - b]
                w[b:e] = np.floor(parts * U32_MAX).astype(np.uint32)
    elif wmode == "zero":
        w = np.zeros(m, dtype=np.uint32)
    elif wmode == "one":
        w = np.full(m, U32_MAX, dtype=np.uint32)
    else:
        w = weights_uniform(m, float(wmode))
    return Graph(n, in_off, in_src, w)


# --- workload definitions (sizes from the paper's Table 3 shapes) -----------

def graph_small_ic(seed: int = 42) -> Graph:
    """R-MAT scale 10: 1,024 vertices, 16,384 edges, IC p = 0.1."""
    return rmat_graph(1024, 16384, seed, "ic0.1")


def graph_lt_scale20(seed: int = 42) -> Graph:
    """R-MAT scale 20: 1,048,576 vertices, 16,777,216 edges, LT 1/in-degree."""
    return rmat_graph(1 << 20, 1 << 24, seed, "lt")


def graph_livejournal_like(seed: int = 42) -> Graph:
    """LiveJournal-shaped R-MAT (4,847,571 vertices, 69M edges), trivalency IC."""
    return rmat_graph(4847571, 69_000_000, seed, "trivalency", levels=23)


def graph_livejournal_like_both(seed: int = 42) -> dict:
    """The LiveJournal-shaped topology once, with two weightings sharing it:
    "trivalency" (IC) and "wc" (IC weighted cascade, 1/in-degree)."""
    src, dst = rmat_edges(4847571, 69_000_000, seed=seed, levels=23)
    in_off, in_src = in_csr(4847571, src, dst)
    return {"trivalency": Graph(4847571, in_off, in_src, weights_trivalency(69_000_000, seed)),
            "wc": Graph(4847571, in_off, in_src, weights_inverse_indegree(in_off))}


def graph_orkut_like(seed: int = 42) -> Graph:
    """Orkut-shaped R-MAT (3,072,441 vertices, 234,369,798 edges), IC p = 0.01."""
    return rmat_graph(3072441, 234_369_798, seed, "ic0.01", levels=22)


# --- many queries: the batched mix and the served arrival trace -------------

BATCH_SCALES = tuple(range(12, 19))


def batched_graph(scale: int, seed: int = 42) -> Graph:
    """R-MAT graph of the batched mix: 2^scale vertices, edge factor 16, weights
    1/in-degree (LT weights, and the weighted-cascade IC probabilities)."""
    return rmat_graph(1 << scale, 16 << scale, seed, "lt")


@dataclass
class QuerySpec:
    """One influence-maximization query of a synthetic workload."""
    graph: str          # "rmat<scale>" or "orkut"
    model: int          # 0 IC, 1 LT
    k: int
    theta: int
    seed: int
    arrival_s: float = 0.0


def batched_queries(nq: int = 256, seed: int = 42) -> list[QuerySpec]:
    """The batched mix: per query a scale uniform in 12..18, IC or LT with
    probability 1/2 each, k uniform in [5, 100], theta uniform in
    [2^14, 2^20] and its own Philox seed (numpy PCG64 draws keyed by seed)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x717565727921))
    out = []
    for q in range(nq):
        scale = int(rng.integers(12, 19))
        model = int(rng.integers(0, 2))
        k = int(rng.integers(5, 101))
        theta = int(rng.integers(1 << 14, (1 << 20) + 1))
        qseed = (seed ^ ((q + 1) * 0x9E3779B97F4A7C15)) & ((1 << 64) - 1)
        out.append(QuerySpec(f"rmat{scale}", model, k, theta, qseed))
    return out


def served_trace(nq: int = 512, seed: int = 42, rate_per_s: float = 200.0,
                 orkut_frac: float = 0.05) -> list[QuerySpec]:
    """Poisson arrivals (exponential gaps, mean 1/rate) of queries drawn like
    the batched mix; a fraction orkut_frac of them runs on the Orkut-shaped
    graph (IC p = 0.01) with theta uniform in [2^6, 2^10] (the mix's range
    divided by 256: an Orkut-shaped RRR set averages ~6e4 members)."""
    base = batched_queries(nq, seed + 1)
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x6172726976616c))
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=nq))
    for q, spec in enumerate(base):
        spec.arrival_s = float(t[q])
        if rng.random() < orkut_frac:
            spec.graph = "orkut"
            spec.model = 0
            spec.theta = int(rng.integers(1 << 6, (1 << 10) + 1))
    return base
