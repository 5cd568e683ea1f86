"""Thin ctypes binding over libim.so (C ABI in include/im.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host), torch tensors (host or CUDA) or
raw integer addresses; streams may be None (torch's current stream when
torch has CUDA, else the legacy default stream), a torch.cuda.Stream or a raw
cudaStream_t address.  The library must be built (build.build_library());
loading fails loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

IM_OK = 0
IM_ERR_INVALID_ARG = -1
IM_ERR_OOM = -2
IM_ERR_CUDA = -3
IM_ERR_TIMEOUT = -4
IM_ERR_CAPACITY = -5
IM_ERR_BUSY = -6
IM_ERR_UNSUPPORTED = -7

IM_IC, IM_LT = 0, 1
IM_GREEDY_PLAIN, IM_RANDGREEDI, IM_GREEDY_LAZY = 0, 1, 2
IM_AGG_STREAM, IM_AGG_GREEDY = 0, 1


class ImError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class CoverOpts(ctypes.Structure):
    """im_cover_opts (see include/im.h)."""
    _fields_ = [("algo", ctypes.c_int32), ("partitions", ctypes.c_int32),
                ("alpha_num", ctypes.c_int32), ("alpha_den", ctypes.c_int32),
                ("delta", ctypes.c_double), ("partition_seed", ctypes.c_uint64),
                ("fused", ctypes.c_int32), ("aggregator", ctypes.c_int32)]


def cover_opts(algo: int = IM_GREEDY_PLAIN, partitions: int = 148, alpha: tuple = (1, 1),
               delta: float = 0.077, partition_seed: int = 42, fused: bool = True,
               aggregator: int = IM_AGG_STREAM) -> CoverOpts:
    return CoverOpts(algo, partitions, alpha[0], alpha[1], delta, partition_seed, int(fused),
                     aggregator)


_LIB = None


def lib():
    """Load libim.so (must already be built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libim.so is not built ({path}); run "
                               "paper_2408_10982_gb300.build.build_library()")
        L = ctypes.CDLL(path)
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        pp = ctypes.POINTER(ctypes.c_void_p)
        sigs = {
            "im_status_str": ([ctypes.c_int], ctypes.c_char_p),
            "im_last_error": ([], ctypes.c_char_p),
            "im_device_info": ([vp, vp], ctypes.c_int),
            "im_trim_memory": ([], ctypes.c_int),
            "im_graph_create": ([vp, vp, vp, i64, i64, vp, pp], ctypes.c_int),
            "im_graph_destroy": ([vp], ctypes.c_int),
            "im_graph_info": ([vp, vp, vp, vp], ctypes.c_int),
            "im_pool_create": ([vp, i64, i64, pp], ctypes.c_int),
            "im_pool_destroy": ([vp], ctypes.c_int),
            "im_pool_reset": ([vp], ctypes.c_int),
            "im_pool_info": ([vp, vp, vp, vp], ctypes.c_int),
            "im_sample_rrr": ([vp, ctypes.c_int, u64, u64, u64, vp, vp], ctypes.c_int),
            "im_pool_export": ([vp, vp, vp, vp], ctypes.c_int),
            "im_pool_index": ([vp, vp], ctypes.c_int),
            "im_index_export": ([vp, vp, vp, vp], ctypes.c_int),
            "im_max_k_cover": ([vp, i32, vp, vp, vp, vp, vp, vp], ctypes.c_int),
            "im_randgreedi_details": ([vp] + [vp] * 12 + [vp], ctypes.c_int),
            "im_partition": ([i64, i32, u64, vp, vp], ctypes.c_int),
            "im_pool_sample_bytes": ([vp, vp], ctypes.c_int),
            "im_randgreedi_stats": ([vp, vp, vp], ctypes.c_int),
            "im_greedy_stats": ([vp, vp], ctypes.c_int),
            "im_max_k_cover_noalloc": ([vp, vp, vp, vp, i64, i64, i32, vp, vp, vp, vp, vp],
                                       ctypes.c_int),
            "im_pool_reserve": ([vp, i64, i64], ctypes.c_int),
            "im_batch_create": ([pp], ctypes.c_int),
            "im_server_create": ([vp, pp], ctypes.c_int),
            "im_server_destroy": ([vp], ctypes.c_int),
            "im_server_submit": ([vp, vp, vp], ctypes.c_int),
            "im_server_poll": ([vp, ctypes.c_uint64, vp, vp, vp, vp], ctypes.c_int),
            "im_server_wait": ([vp, ctypes.c_uint64, ctypes.c_double, vp, vp, vp, vp], ctypes.c_int),
            "im_server_stats": ([vp, vp, vp, vp], ctypes.c_int),
            "im_batch_destroy": ([vp], ctypes.c_int),
            "im_spread": ([vp, ctypes.c_int, vp, i32, u64, u64, u64, vp, vp, vp, vp], ctypes.c_int),
            "im_autotune": ([vp, ctypes.c_int, u64, i64, i32, vp, vp, vp], ctypes.c_int),
            "im_solve_batch": ([vp, vp, i32, i32, vp, vp, vp, vp], ctypes.c_int),
            "im_solve": ([vp, ctypes.c_int, i32, ctypes.c_double, ctypes.c_double, u64, vp, vp,
                          vp, vp, vp, vp, vp], ctypes.c_int),
            "im_opim": ([vp, ctypes.c_int, i32, ctypes.c_double, ctypes.c_double, u64, i64, vp,
                         vp, vp, vp, vp], ctypes.c_int),
            "im_tune_set": ([i32, i64], ctypes.c_int),
            "im_tune_get": ([i32, vp], ctypes.c_int),
            "im_profile_enable": ([i32], ctypes.c_int),
            "im_profile_reset": ([], ctypes.c_int),
            "im_profile_read": ([i32, vp, vp, vp, vp], ctypes.c_int),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = L
    return _LIB


def status_str(s: int) -> str:
    return lib().im_status_str(s).decode()


def last_error() -> str:
    return lib().im_last_error().decode()


def _check(st: int, what: str):
    if st != IM_OK:
        raise ImError(st, f"{what}: {status_str(st)} ({last_error()})")


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as an array")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# --- one function per C entry point (same names, same argument order) -------

def im_device_info():
    sms, dev = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().im_device_info(ctypes.byref(sms), ctypes.byref(dev)), "im_device_info")
    return sms.value, dev.value


def im_trim_memory():
    _check(lib().im_trim_memory(), "im_trim_memory")


def im_graph_create(in_off, in_src, w, n: int, m: int, stream=None):
    h = ctypes.c_void_p()
    _check(lib().im_graph_create(_ptr(in_off), _ptr(in_src), _ptr(w), n, m, _stream(stream),
                                 ctypes.byref(h)), "im_graph_create")
    return h


def im_graph_destroy(g):
    _check(lib().im_graph_destroy(g), "im_graph_destroy")


def im_graph_info(g):
    n, m, lt = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib().im_graph_info(g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(lt)),
           "im_graph_info")
    return n.value, m.value, lt.value


def im_pool_create(g, max_sets: int, max_entries: int):
    h = ctypes.c_void_p()
    _check(lib().im_pool_create(g, max_sets, max_entries, ctypes.byref(h)), "im_pool_create")
    return h


def im_pool_destroy(p):
    _check(lib().im_pool_destroy(p), "im_pool_destroy")


def im_pool_reset(p):
    _check(lib().im_pool_reset(p), "im_pool_reset")


def im_pool_info(p):
    t, T, e = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().im_pool_info(p, ctypes.byref(t), ctypes.byref(T), ctypes.byref(e)),
           "im_pool_info")
    return t.value, T.value, e.value


def im_sample_rrr(g, model: int, seed: int, first_sample_id: int, num_samples: int, pool,
                  stream=None):
    _check(lib().im_sample_rrr(g, model, seed, first_sample_id, num_samples, pool,
                               _stream(stream)), "im_sample_rrr")


def im_pool_export(p, set_off, members, stream=None):
    _check(lib().im_pool_export(p, _ptr(set_off), _ptr(members), _stream(stream)),
           "im_pool_export")


def im_pool_index(p, stream=None):
    _check(lib().im_pool_index(p, _stream(stream)), "im_pool_index")


def im_index_export(p, vtx_off, set_ids, stream=None):
    _check(lib().im_index_export(p, _ptr(vtx_off), _ptr(set_ids), _stream(stream)),
           "im_index_export")


def im_max_k_cover(p, k: int, opts: CoverOpts | None, seeds, gains, num_seeds, coverage,
                   stream=None):
    _check(lib().im_max_k_cover(p, k, None if opts is None else ctypes.byref(opts), _ptr(seeds),
                                _ptr(gains), _ptr(num_seeds), _ptr(coverage), _stream(stream)),
           "im_max_k_cover")


def im_randgreedi_details(p, local_seeds=None, local_gains=None, local_n=None, local_cov=None,
                          thr=None, bucket_cov=None, bucket_n=None, bucket_seeds=None,
                          bucket_gains=None, stream=None):
    P, B, ch = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().im_randgreedi_details(
        p, ctypes.byref(P), ctypes.byref(B), _ptr(local_seeds), _ptr(local_gains), _ptr(local_n),
        _ptr(local_cov), _ptr(thr), _ptr(bucket_cov), _ptr(bucket_n), _ptr(bucket_seeds),
        _ptr(bucket_gains), ctypes.byref(ch), _stream(stream)), "im_randgreedi_details")
    return P.value, B.value, ch.value


def im_partition(n: int, P: int, partition_seed: int, part, stream=None):
    _check(lib().im_partition(n, P, partition_seed, _ptr(part), _stream(stream)), "im_partition")


def im_max_k_cover_noalloc(set_off, members, vtx_off, set_ids, n: int, theta: int, k: int,
                           seeds, gains, num_seeds, coverage, stream=None):
    """Greedy max-k-cover over caller-owned device arrays, allocating nothing."""
    _check(lib().im_max_k_cover_noalloc(_ptr(set_off), _ptr(members), _ptr(vtx_off),
                                        _ptr(set_ids), n, theta, k, _ptr(seeds), _ptr(gains),
                                        _ptr(num_seeds), _ptr(coverage), _stream(stream)),
           "im_max_k_cover_noalloc")


class SolveInfo(ctypes.Structure):
    """im_solve_info (see include/im.h)."""
    _fields_ = [("rounds", ctypes.c_int32), ("keep_pools", ctypes.c_int32),
                ("theta_rounds", ctypes.c_int64 * 64), ("cov_rounds", ctypes.c_int64 * 64),
                ("lb", ctypes.c_double), ("theta", ctypes.c_int64),
                ("round_entries", ctypes.c_int64), ("final_entries", ctypes.c_int64),
                ("examined", ctypes.c_int64), ("round_pool", ctypes.c_void_p),
                ("final_pool", ctypes.c_void_p)]


class OpimInfo(ctypes.Structure):
    """im_opim_info (see include/im.h)."""
    _fields_ = [("rounds", ctypes.c_int32), ("keep_pools", ctypes.c_int32),
                ("theta", ctypes.c_int64 * 64), ("cov1", ctypes.c_int64 * 64),
                ("cov2", ctypes.c_int64 * 64), ("cov1_upper", ctypes.c_int64 * 64),
                ("alpha", ctypes.c_double * 64), ("sigma_lower", ctypes.c_double),
                ("sigma_upper", ctypes.c_double), ("guarantee", ctypes.c_double),
                ("theta_max", ctypes.c_double), ("theta0", ctypes.c_int64),
                ("max_rounds", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("a", ctypes.c_double), ("r1_pool", ctypes.c_void_p),
                ("r2_pool", ctypes.c_void_p)]


def im_opim(g, model: int, k: int, eps: float, delta: float, seed: int, theta_cap: int = 0,
            opts: CoverOpts | None = None, stream=None, keep_pools: bool = False):
    """OPIM rounds with GreediRIS seed selection: returns (seeds, info).  With
    keep_pools, info.r1_pool / info.r2_pool must be destroyed by the caller."""
    seeds = np.zeros(k, np.int32)
    ns = ctypes.c_int32()
    info = OpimInfo()
    info.keep_pools = 1 if keep_pools else 0
    _check(lib().im_opim(g, model, k, eps, delta, seed, theta_cap,
                         None if opts is None else ctypes.byref(opts), seeds.ctypes.data,
                         ctypes.byref(ns), ctypes.byref(info), _stream(stream)), "im_opim")
    return seeds[: ns.value].copy(), info


class Query(ctypes.Structure):
    """im_query (see include/im.h)."""
    _fields_ = [("graph", ctypes.c_void_p), ("model", ctypes.c_int32), ("k", ctypes.c_int32),
                ("theta", ctypes.c_int64), ("seed", ctypes.c_uint64), ("cover", CoverOpts)]


class Result(ctypes.Structure):
    """im_result (see include/im.h)."""
    _fields_ = [("num_seeds", ctypes.c_int32), ("status", ctypes.c_int32),
                ("coverage", ctypes.c_int64), ("entries", ctypes.c_int64),
                ("partitions", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def im_batch_create():
    h = ctypes.c_void_p()
    _check(lib().im_batch_create(ctypes.byref(h)), "im_batch_create")
    return h


def im_batch_destroy(b):
    _check(lib().im_batch_destroy(b), "im_batch_destroy")


def im_solve_batch(b, queries, kmax: int, stream=None, with_partitions: bool = False):
    """queries: list of (graph handle, model, k, theta, seed[, CoverOpts]).
    Returns a list of (seeds, gains, coverage, entries) per query, with the
    partition count a RandGreedi query used appended when with_partitions."""
    nq = len(queries)

    def q(t):
        g, m, k, th, sd = t[:5]
        opts = t[5] if len(t) > 5 and t[5] is not None else CoverOpts()
        return Query(g.value if hasattr(g, "value") else g, m, k, th, sd, opts)
    arr = (Query * nq)(*[q(t) for t in queries])
    seeds = np.zeros(nq * kmax, np.int32)
    gains = np.zeros(nq * kmax, np.int64)
    res = (Result * nq)()
    _check(lib().im_solve_batch(b, arr, nq, kmax, seeds.ctypes.data, gains.ctypes.data, res,
                                _stream(stream)), "im_solve_batch")
    out = []
    for i in range(nq):
        m = res[i].num_seeds
        r = (seeds[i * kmax:i * kmax + m].copy(), gains[i * kmax:i * kmax + m].copy(),
             res[i].coverage, res[i].entries)
        out.append(r + (res[i].partitions,) if with_partitions else r)
    return out


def im_spread(g, model: int, seeds, seed: int, first_run: int, runs: int, activated=None,
              root_hit=None, stream=None) -> int:
    """Forward simulation of runs first_run .. first_run+runs-1 from `seeds`
    (host numpy / torch, host or device); fills `activated` int64[runs] and
    `root_hit` uint8[runs] when given; returns the total activated count."""
    sd = np.ascontiguousarray(seeds, dtype=np.int32) if isinstance(seeds, (list, tuple, np.ndarray)) \
        else seeds
    total = ctypes.c_int64()
    _check(lib().im_spread(g.value if hasattr(g, "value") else g, model, _ptr(sd), len(sd), seed,
                           first_run, runs, _ptr(activated), _ptr(root_hit), ctypes.byref(total),
                           _stream(stream)), "im_spread")
    return total.value


class TuneResult(ctypes.Structure):
    """im_tune_result (see include/im.h)."""
    _fields_ = [("lt_group", ctypes.c_int32), ("index_replicas", ctypes.c_int32),
                ("rg_evals", ctypes.c_int32), ("rg_cluster", ctypes.c_int32),
                ("lt_cache", ctypes.c_int32), ("greedy_hot", ctypes.c_int32),
                ("ms", (ctypes.c_double * 8) * 6)]


def im_autotune(g, model: int, seed: int, theta: int, k: int, rg_opts: CoverOpts | None = None,
                stream=None) -> dict:
    """Time the result-invariant knobs on a probe of the workload and keep the
    fastest values; returns the chosen values and the measured times."""
    r = TuneResult()
    _check(lib().im_autotune(g.value if hasattr(g, "value") else g, model, seed, theta, k,
                             None if rg_opts is None else ctypes.byref(rg_opts), ctypes.byref(r),
                             _stream(stream)), "im_autotune")
    return {"lt_group": r.lt_group, "index_replicas": r.index_replicas, "rg_evals": r.rg_evals,
            "rg_cluster": r.rg_cluster, "lt_cache": r.lt_cache, "greedy_hot": r.greedy_hot,
            "ms": [[round(x, 3) for x in row] for row in r.ms]}


class ServerOpts(ctypes.Structure):
    """im_server_opts (see include/im.h)."""
    _fields_ = [("workers", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("mem_budget", ctypes.c_int64), ("heavy_members", ctypes.c_int64)]


def im_server_create(workers: int = 2, max_batch: int = 256, mem_budget: int = 64 << 30,
                     heavy_members: int = 0):
    h = ctypes.c_void_p()
    o = ServerOpts(workers, max_batch, mem_budget, heavy_members)
    _check(lib().im_server_create(ctypes.byref(o), ctypes.byref(h)), "im_server_create")
    return h


def im_server_destroy(s):
    _check(lib().im_server_destroy(s), "im_server_destroy")


def im_server_submit(s, graph, model: int, k: int, theta: int, seed: int,
                     opts: CoverOpts | None = None) -> int:
    q = Query(graph.value if hasattr(graph, "value") else graph, model, k, theta, seed,
              opts if opts is not None else CoverOpts())
    t = ctypes.c_uint64()
    _check(lib().im_server_submit(s, ctypes.byref(q), ctypes.byref(t)), "im_server_submit")
    return t.value


def im_server_wait(s, ticket: int, kmax: int, timeout_s: float = 600.0):
    """(seeds, coverage, latency ms) of a request, blocking until it is done."""
    seeds = np.zeros(max(kmax, 1), np.int32)
    ns = ctypes.c_int32()
    cov = ctypes.c_int64()
    lat = ctypes.c_double()
    _check(lib().im_server_wait(s, ticket, timeout_s, seeds.ctypes.data, ctypes.byref(ns),
                                ctypes.byref(cov), ctypes.byref(lat)), "im_server_wait")
    return seeds[: ns.value].copy(), cov.value, lat.value


def im_server_poll(s, ticket: int, kmax: int):
    """None while pending, else (seeds, coverage, latency ms)."""
    seeds = np.zeros(max(kmax, 1), np.int32)
    ns = ctypes.c_int32()
    cov = ctypes.c_int64()
    lat = ctypes.c_double()
    st = lib().im_server_poll(s, ticket, seeds.ctypes.data, ctypes.byref(ns), ctypes.byref(cov),
                              ctypes.byref(lat))
    if st == IM_ERR_BUSY:
        return None
    _check(st, "im_server_poll")
    return seeds[: ns.value].copy(), cov.value, lat.value


def im_server_stats(s):
    b, q, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().im_server_stats(s, ctypes.byref(b), ctypes.byref(q), ctypes.byref(w)),
           "im_server_stats")
    return b.value, q.value, w.value


def im_pool_reserve(p, max_sets: int, max_entries: int):
    _check(lib().im_pool_reserve(p, max_sets, max_entries), "im_pool_reserve")


def im_solve(g, model: int, k: int, eps: float, ell: float, seed: int,
             opts: CoverOpts | None = None, stream=None, keep_pools: bool = False):
    """IMM (Alg. 1) on the device path: returns (seeds, coverage, theta, info).
    With keep_pools, info.round_pool / info.final_pool are pool handles the
    caller must destroy (im_pool_destroy)."""
    seeds = np.zeros(k, np.int32)
    ns = ctypes.c_int32()
    cov = ctypes.c_int64()
    theta = ctypes.c_int64()
    info = SolveInfo()
    info.keep_pools = 1 if keep_pools else 0
    _check(lib().im_solve(g, model, k, eps, ell, seed,
                          None if opts is None else ctypes.byref(opts), seeds.ctypes.data,
                          ctypes.byref(ns), ctypes.byref(cov), ctypes.byref(theta),
                          ctypes.byref(info), _stream(stream)), "im_solve")
    return seeds[: ns.value].copy(), cov.value, theta.value, info


def im_randgreedi_stats(p, P: int, B: int, stream=None) -> np.ndarray:
    out = np.zeros((P + B) * 6, np.int64)
    _check(lib().im_randgreedi_stats(p, out.ctypes.data, _stream(stream)), "im_randgreedi_stats")
    return out.reshape(P + B, 6)


def im_greedy_stats(p) -> dict:
    """The pool's last lazy-greedy cover: rounds, candidate evaluations,
    covering-subset entries they scanned, builds of the sorted bound list."""
    out = np.zeros(4, np.int64)
    _check(lib().im_greedy_stats(p, out.ctypes.data), "im_greedy_stats")
    return dict(rounds=int(out[0]), evals=int(out[1]), scanned=int(out[2]), builds=int(out[3]))


def im_pool_sample_bytes(p) -> int:
    b = ctypes.c_int64()
    _check(lib().im_pool_sample_bytes(p, ctypes.byref(b)), "im_pool_sample_bytes")
    return b.value


IM_TUNE_LT_GROUP = 0
IM_TUNE_RG_CLUSTER = 1
IM_TUNE_INDEX_REPLICAS = 2
IM_TUNE_RG_EVALS = 3
IM_TUNE_GREEDY_EVALS = 4
IM_TUNE_LT_CACHE = 5
IM_TUNE_GREEDY_HOT = 6


def im_tune_set(knob: int, value: int):
    _check(lib().im_tune_set(knob, value), "im_tune_set")


def im_tune_get(knob: int) -> int:
    v = ctypes.c_int64()
    _check(lib().im_tune_get(knob, ctypes.byref(v)), "im_tune_get")
    return v.value


def im_profile_enable(on: bool = True):
    _check(lib().im_profile_enable(int(on)), "im_profile_enable")


def im_profile_reset():
    _check(lib().im_profile_reset(), "im_profile_reset")


def im_profile_read(max_entries: int = 64) -> dict:
    """{kernel name: (launches, total ms)} since the last reset."""
    names = ctypes.create_string_buffer(48 * max_entries)
    launches = np.zeros(max_entries, np.int64)
    ms = np.zeros(max_entries, np.float64)
    cnt = ctypes.c_int32()
    _check(lib().im_profile_read(max_entries, names, launches.ctypes.data, ms.ctypes.data,
                                 ctypes.byref(cnt)), "im_profile_read")
    raw = names.raw
    out = {}
    for i in range(cnt.value):
        name = raw[48 * i:48 * (i + 1)].split(b"\0", 1)[0].decode()
        out[name] = (int(launches[i]), float(ms[i]))
    return out


# --- convenience wrappers (still only marshalling) ---------------------------

class Graph:
    """Owns an im_graph built from an inputs.Graph (host arrays)."""

    def __init__(self, g, stream=None):
        self.n, self.m = int(g.n), int(g.m)
        self.handle = im_graph_create(np.ascontiguousarray(g.in_off, np.int64),
                                      np.ascontiguousarray(g.in_src, np.int32),
                                      np.ascontiguousarray(g.w, np.uint32), self.n, self.m, stream)

    def close(self):
        if self.handle is not None:
            im_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class CoverResult:
    seeds: np.ndarray
    gains: np.ndarray
    coverage: int


class Pool:
    """Owns an im_pool; numpy in, numpy out."""

    def __init__(self, graph: Graph, max_sets: int, max_entries: int):
        self.graph = graph
        self.handle = im_pool_create(graph.handle, max_sets, max_entries)

    def sample(self, model: int, seed: int, first: int, count: int, stream=None):
        im_sample_rrr(self.graph.handle, model, seed, first, count, self.handle, stream)

    def info(self):
        return im_pool_info(self.handle)

    def sample_bytes(self) -> int:
        return im_pool_sample_bytes(self.handle)

    def reset(self):
        im_pool_reset(self.handle)

    def export(self, stream=None):
        theta, total, _ = self.info()
        set_off = np.zeros(theta + 1, np.int64)
        members = np.zeros(max(total, 1), np.int32)
        im_pool_export(self.handle, set_off, members, stream)
        return set_off, members[:total]

    def index(self, stream=None):
        theta, total, _ = self.info()
        vtx_off = np.zeros(self.graph.n + 1, np.int64)
        set_ids = np.zeros(max(total, 1), np.int32)
        im_index_export(self.handle, vtx_off, set_ids, stream)
        return vtx_off, set_ids[:total]

    def cover(self, k: int, opts: CoverOpts | None = None, stream=None) -> CoverResult:
        seeds = np.zeros(k, np.int32)
        gains = np.zeros(k, np.int64)
        ns = np.zeros(1, np.int32)
        cov = np.zeros(1, np.int64)
        im_max_k_cover(self.handle, k, opts, seeds, gains, ns, cov, stream)
        return CoverResult(seeds[: ns[0]].copy(), gains[: ns[0]].copy(), int(cov[0]))

    def randgreedi_details(self, k: int, P: int, B: int, stream=None) -> dict:
        d = dict(local_seeds=np.zeros(P * k, np.int32), local_gains=np.zeros(P * k, np.int64),
                 local_n=np.zeros(P, np.int32), local_cov=np.zeros(P, np.int64),
                 thr=np.zeros(B, np.int64), bucket_cov=np.zeros(B, np.int64),
                 bucket_n=np.zeros(B, np.int32), bucket_seeds=np.zeros(B * k, np.int32),
                 bucket_gains=np.zeros(B * k, np.int64))
        P2, B2, chosen = im_randgreedi_details(self.handle, stream=stream, **d)
        assert (P2, B2) == (P, B)
        d["local_seeds"] = d["local_seeds"].reshape(P, k)
        d["local_gains"] = d["local_gains"].reshape(P, k)
        d["bucket_seeds"] = d["bucket_seeds"].reshape(B, k)
        d["bucket_gains"] = d["bucket_gains"].reshape(B, k)
        d["chosen"] = chosen
        return d

    def close(self):
        if self.handle is not None:
            im_pool_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
