"""ctypes wrapper around oracle.c -- TEST INFRASTRUCTURE ONLY.

Each function below follows the paper passage cited in oracle.c; this file
only marshals numpy arrays.  The shared object is compiled with gcc on first
use (and by `__graft_entry__.build()`).

Parity status (what pins each function, see tests/test_oracle_*.py):
  philox        known-answer vectors + cuRAND's host Philox generator
  root          chi-square uniformity; root always in its own set
  sample (IC)   equals reverse reachability in the explicit live-edge world
                (scipy BFS); exact inclusion probabilities by enumeration
  sample (LT)   equals the backward pick chain of the explicit world; simple
                path; exact inclusion probabilities by enumeration
  invert        dict-of-sets transpose
  greedy        from-scratch marginal-gain greedy with Python sets;
                (1-1/e) and truncated (1-(1-1/k)^j) bounds vs optimal cover
  lazy_greedy   equals the standard greedy (submodularity: stale gains are
                upper bounds) on random and tie-heavy instances; a
                hand-worked heap trace of Alg. 2
  partition     chi-square balance; determinism
  stream        (1/2)/(1+delta) bound vs the optimal cover of the stream
  randgreedi    locals equal greedy on the induced instance; final rule;
                naive global step equals the standard greedy over the
                gathered seeds
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_LIB = None

IC, LT = 0, 1

c_i64p = ctypes.POINTER(ctypes.c_int64)
c_i32p = ctypes.POINTER(ctypes.c_int32)


def build() -> str:
    """Compile oracle.c into a shared object next to it (idempotent)."""
    if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = f"{_SO}.{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        vp, i64, u64, i32, u32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_int32, ctypes.c_uint32)
        lib.orc_philox.argtypes = [vp, vp, vp]
        lib.orc_root.restype = u32
        lib.orc_root.argtypes = [u64, u32, i64]
        lib.orc_ic_coin.restype = u32
        lib.orc_ic_coin.argtypes = [u64, u32, i64]
        lib.orc_lt_draw.restype = u32
        lib.orc_lt_draw.argtypes = [u64, u32, u32]
        lib.orc_part_of.restype = i32
        lib.orc_part_of.argtypes = [u64, u32, i32]
        lib.orc_partition.argtypes = [i64, i32, u64, vp]
        lib.orc_sample.restype = ctypes.c_int
        lib.orc_sample.argtypes = [ctypes.c_int, i64, vp, vp, vp, u64, u64, u64, ctypes.c_int,
                                   ctypes.POINTER(c_i64p), ctypes.POINTER(c_i32p), vp, vp]
        lib.orc_free.argtypes = [vp]
        lib.orc_invert.restype = ctypes.c_int
        lib.orc_invert.argtypes = [i64, i64, vp, vp, vp, vp]
        lib.orc_greedy.restype = ctypes.c_int
        lib.orc_greedy.argtypes = [i64, i64, vp, vp, vp, vp, i32, vp, i64, vp, vp, vp, vp]
        lib.orc_num_buckets.restype = i32
        lib.orc_num_buckets.argtypes = [i32, ctypes.c_double]
        lib.orc_bucket_thresholds.argtypes = [i64, i32, ctypes.c_double, i32, vp]
        lib.orc_stream_buckets.restype = ctypes.c_int
        lib.orc_stream_buckets.argtypes = [i64, vp, vp, vp, i64, i32, i32, vp, vp, vp, vp, vp]
        lib.orc_spread.restype = ctypes.c_int
        lib.orc_spread.argtypes = [ctypes.c_int, i64, vp, vp, vp, u64, u64, u64, vp, i32, vp, vp]
        lib.orc_randgreedi.restype = ctypes.c_int
        lib.orc_randgreedi.argtypes = [i64, i64, vp, vp, vp, vp, i32, i32, u64, i32,
                                       ctypes.c_double, i32] + [vp] * 14
        lib.orc_lazy_greedy.restype = ctypes.c_int
        lib.orc_lazy_greedy.argtypes = [i64, i64, vp, vp, i32, vp, i64, vp, vp, vp, vp]
        _LIB = lib
    return _LIB


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --- random stream -----------------------------------------------------------

def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under a 2-word key."""
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _lib().orc_philox(_p(c), _p(k), _p(out))
    return out


def root(seed: int, s: int, n: int) -> int:
    return int(_lib().orc_root(seed, s, n))


def ic_coin(seed: int, s: int, e: int) -> int:
    return int(_lib().orc_ic_coin(seed, s, e))


def lt_draw(seed: int, s: int, v: int) -> int:
    return int(_lib().orc_lt_draw(seed, s, v))


def partition(n: int, P: int, pseed: int) -> np.ndarray:
    part = np.zeros(n, dtype=np.int32)
    _lib().orc_partition(n, P, pseed, _p(part))
    return part


# --- sampling ---------------------------------------------------------------

@dataclass
class Pool:
    """RRR sets in CSR by sample id (set_off int64[theta+1], members int32[T])."""
    set_off: np.ndarray
    members: np.ndarray
    examined: int

    @property
    def theta(self) -> int:
        return int(self.set_off.shape[0] - 1)

    def set(self, i: int) -> np.ndarray:
        return self.members[self.set_off[i]:self.set_off[i + 1]]


def sample(model: int, graph, seed: int, first: int, count: int,
           keep_order: bool = False) -> Pool:
    """RRR sets for sample ids first .. first+count-1 (IC = 0, LT = 1)."""
    if first + count > 1 << 32:
        raise ValueError("sample ids must stay below 2^32")
    in_off = _c(graph.in_off, np.int64)
    in_src = _c(graph.in_src, np.int32)
    w = _c(graph.w, np.uint32)
    so = c_i64p()
    mem = c_i32p()
    total = ctypes.c_int64()
    examined = ctypes.c_int64()
    rc = _lib().orc_sample(model, graph.n, _p(in_off), _p(in_src), _p(w), seed, first, count,
                           int(keep_order), ctypes.byref(so), ctypes.byref(mem),
                           ctypes.byref(total), ctypes.byref(examined))
    if rc != 0:
        raise MemoryError("oracle sampling ran out of memory")
    set_off = np.ctypeslib.as_array(so, shape=(count + 1,)).copy()
    members = (np.ctypeslib.as_array(mem, shape=(total.value,)).copy()
               if total.value else np.zeros(0, dtype=np.int32))
    _lib().orc_free(ctypes.cast(so, ctypes.c_void_p))
    _lib().orc_free(ctypes.cast(mem, ctypes.c_void_p))
    return Pool(set_off, members, int(examined.value))


# --- covering subsets and greedy --------------------------------------------

def invert(n: int, pool: Pool) -> tuple[np.ndarray, np.ndarray]:
    """Covering subsets S(v) as CSR (vtx_off int64[n+1], set_ids int32[T])."""
    vtx_off = np.zeros(n + 1, dtype=np.int64)
    set_ids = np.zeros(max(1, pool.members.shape[0]), dtype=np.int32)
    if _lib().orc_invert(n, pool.theta, _p(pool.set_off), _p(pool.members), _p(vtx_off),
                         _p(set_ids)):
        raise MemoryError
    return vtx_off, set_ids[: pool.members.shape[0]]


@dataclass
class Cover:
    seeds: np.ndarray
    gains: np.ndarray
    coverage: int


def greedy(n: int, pool: Pool, inv, k: int, cand: np.ndarray | None = None) -> Cover:
    """Plain greedy max-k-cover (ties -> smallest id, stops at zero gain)."""
    vtx_off, set_ids = inv
    seeds = np.zeros(max(k, 1), dtype=np.int32)
    gains = np.zeros(max(k, 1), dtype=np.int64)
    ns = ctypes.c_int32()
    cov = ctypes.c_int64()
    cand_a = None if cand is None else _c(cand, np.int32)
    if cand_a is not None and cand_a.size == 0:      # no candidates, no seeds
        return Cover(np.zeros(0, np.int32), np.zeros(0, np.int64), 0)
    rc = _lib().orc_greedy(n, pool.theta, _p(pool.set_off), _p(pool.members), _p(vtx_off),
                           _p(set_ids), k, _p(cand_a), 0 if cand_a is None else cand_a.size,
                           _p(seeds), _p(gains), ctypes.byref(ns), ctypes.byref(cov))
    if rc:
        raise MemoryError
    return Cover(seeds[: ns.value].copy(), gains[: ns.value].copy(), int(cov.value))


def lazy_greedy(n: int, pool: Pool, inv, k: int, cand: np.ndarray | None = None) -> Cover:
    """Lazy greedy max-k-cover of Alg. 2 (a max heap of stale gains; ties ->
    smallest id, stops at zero gain)."""
    vtx_off, set_ids = inv
    seeds = np.zeros(max(k, 1), dtype=np.int32)
    gains = np.zeros(max(k, 1), dtype=np.int64)
    ns = ctypes.c_int32()
    cov = ctypes.c_int64()
    cand_a = None if cand is None else _c(cand, np.int32)
    if cand_a is not None and cand_a.size == 0:
        return Cover(np.zeros(0, np.int32), np.zeros(0, np.int64), 0)
    rc = _lib().orc_lazy_greedy(n, pool.theta, _p(vtx_off), _p(set_ids), k, _p(cand_a),
                                0 if cand_a is None else cand_a.size, _p(seeds), _p(gains),
                                ctypes.byref(ns), ctypes.byref(cov))
    if rc:
        raise MemoryError
    return Cover(seeds[: ns.value].copy(), gains[: ns.value].copy(), int(cov.value))


def num_buckets(k: int, delta: float) -> int:
    return int(_lib().orc_num_buckets(k, delta))


def bucket_thresholds(l: int, k: int, delta: float) -> np.ndarray:
    B = num_buckets(k, delta)
    thr = np.zeros(B, dtype=np.int64)
    _lib().orc_bucket_thresholds(l, k, delta, B, _p(thr))
    return thr


@dataclass
class Buckets:
    cov: np.ndarray
    n: np.ndarray
    seeds: np.ndarray
    gains: np.ndarray


def stream_buckets(theta: int, inv, stream, k: int, thr: np.ndarray) -> Buckets:
    """Alg. 5 over an explicit stream of vertex ids."""
    vtx_off, set_ids = inv
    st = _c(stream, np.int32)
    B = thr.shape[0]
    thr = _c(thr, np.int64)
    bc = np.zeros(B, dtype=np.int64)
    bn = np.zeros(B, dtype=np.int32)
    bs = np.zeros(B * k, dtype=np.int32)
    bg = np.zeros(B * k, dtype=np.int64)
    if _lib().orc_stream_buckets(theta, _p(vtx_off), _p(set_ids), _p(st), st.size, k, B,
                                 _p(thr), _p(bc), _p(bn), _p(bs), _p(bg)):
        raise MemoryError
    return Buckets(bc, bn, bs.reshape(B, k), bg.reshape(B, k))


@dataclass
class RandGreedi:
    local_seeds: np.ndarray     # [P, k]
    local_gains: np.ndarray     # [P, k]
    local_n: np.ndarray         # [P]
    local_cov: np.ndarray       # [P]
    thr: np.ndarray             # [B]
    buckets: Buckets
    chosen: int                 # -1: best bucket, else the winning partition
    seeds: np.ndarray
    gains: np.ndarray
    coverage: int


def trunc_count(k: int, alpha_num: int, alpha_den: int) -> int:
    """Seeds streamed per partition: ceil(alpha k), at least 1 (Sec. 3.3.2)."""
    return max(1, min(k, -(-k * alpha_num // alpha_den)))


def randgreedi(n: int, pool: Pool, inv, k: int, P: int, pseed: int, trunc: int,
               delta: float, naive: bool = False) -> RandGreedi:
    """Alg. 3 + Alg. 4 with the streaming aggregator of Alg. 5 and truncation
    (Sec. 3.3.2); naive=True: Alg. 4's global step is the lazy greedy of Alg. 2
    over the gathered local seeds, reported as the single bucket 0."""
    vtx_off, set_ids = inv
    B = 1 if naive else num_buckets(k, delta)
    ls = np.zeros(P * k, dtype=np.int32)
    lg = np.zeros(P * k, dtype=np.int64)
    ln = np.zeros(P, dtype=np.int32)
    lc = np.zeros(P, dtype=np.int64)
    thr = np.zeros(B, dtype=np.int64)
    bc = np.zeros(B, dtype=np.int64)
    bn = np.zeros(B, dtype=np.int32)
    bs = np.zeros(B * k, dtype=np.int32)
    bg = np.zeros(B * k, dtype=np.int64)
    chosen = np.zeros(1, dtype=np.int32)
    seeds = np.zeros(k, dtype=np.int32)
    gains = np.zeros(k, dtype=np.int64)
    ns = np.zeros(1, dtype=np.int32)
    cov = np.zeros(1, dtype=np.int64)
    rc = _lib().orc_randgreedi(n, pool.theta, _p(pool.set_off), _p(pool.members), _p(vtx_off),
                               _p(set_ids), k, P, pseed, trunc, delta, int(naive), _p(ls),
                               _p(lg), _p(ln),
                               _p(lc), _p(thr), _p(bc), _p(bn), _p(bs), _p(bg), _p(chosen),
                               _p(seeds), _p(gains), _p(ns), _p(cov))
    if rc:
        raise MemoryError
    return RandGreedi(ls.reshape(P, k), lg.reshape(P, k), ln, lc, thr,
                      Buckets(bc, bn, bs.reshape(B, k), bg.reshape(B, k)), int(chosen[0]),
                      seeds[: ns[0]].copy(), gains[: ns[0]].copy(), int(cov[0]))


# --- approximation ratios stated in the paper (Sec. 3.3) ---------------------

def ratio_randgreedi(alpha: float, beta: float) -> float:
    """Theorem 2: local alpha- and global beta-approximations give ab/(a+b)."""
    return alpha * beta / (alpha + beta)


def ratio_streaming(eps: float, delta: float) -> float:
    """Lemma 1: greedy locals (1-1/e) with (1/2-delta) streaming, minus eps."""
    return ratio_randgreedi(1.0 - np.exp(-1.0), 0.5 - delta) - eps


def ratio_truncated_streaming(alpha: float, eps: float, delta: float) -> float:
    """Lemma 3: truncated locals (1-e^-alpha) with (1/2-delta) streaming, minus eps."""
    return ratio_randgreedi(1.0 - np.exp(-alpha), 0.5 - delta) - eps


# --- forward simulation -------------------------------------------------------

def spread(model: int, graph, seed: int, first: int, runs: int, seeds) -> tuple[np.ndarray, np.ndarray]:
    """Forward simulation from `seeds` in the live-edge worlds of sample ids
    first .. first+runs-1: (activated int64[runs], root_hit uint8[runs])."""
    if first + runs > 1 << 32:
        raise ValueError("run ids must stay below 2^32")
    in_off = _c(graph.in_off, np.int64)
    in_src = _c(graph.in_src, np.int32)
    w = _c(graph.w, np.uint32)
    sd = _c(seeds, np.int32)
    act = np.zeros(runs, np.int64)
    hit = np.zeros(runs, np.uint8)
    rc = _lib().orc_spread(model, graph.n, _p(in_off), _p(in_src), _p(w), seed, first, runs,
                           _p(sd), len(sd), _p(act), _p(hit))
    if rc != 0:
        raise MemoryError("oracle spread ran out of memory")
    return act, hit
