"""OPIM driver over the oracle's sampling and covers -- TEST INFRASTRUCTURE ONLY.

The paper runs GreediRIS inside OPIM (Tang et al. 2018; Sec. 3.3.2, Sec. 4.4,
Table 6): every round's samples are split into a selection half R1 and a
validation half R2; seeds selected on R1 (standard greedy, or RandGreedi with
truncation) are scored on R2, and the round reports an instance-wise
approximation guarantee alpha = sigma_l(S) / sigma_u(OPT).  OPIM-C's steps,
in order:
  theta_0 sets in each half (ids: R1 from 0, R2 from 2^31), rounds i = 1 ..
  i_max: select S on R1 (coverage cov1); cov2 = sets of R2 that contain a
  seed (the RIS estimate); an upper bound on the optimal k-set's coverage of
  R1, cov1u = cov1 + the k largest marginal gains |S1(v) \\ C1(S)| (valid for
  any S by submodularity); sigma_l from cov2, sigma_u from cov1u
  (orc_opim_* in oracle.c); stop when alpha >= 1 - 1/e - eps or at i_max,
  else double both halves (appending ids).
The formulas are pinned in tests/test_oracle_opim.py against the tail
equations they solve and against exact spreads of tiny graphs.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import oracle as O

R2_FIRST = 1 << 31


def _lib():
    lib = O._lib()
    if not hasattr(lib, "_opim_ready"):
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int32
        lib.orc_opim_constants.argtypes = [i64, i32, d, d, i64, ctypes.c_void_p]
        lib.orc_opim_lower.restype = d
        lib.orc_opim_lower.argtypes = [i64, i64, i64, d]
        lib.orc_opim_upper.restype = d
        lib.orc_opim_upper.argtypes = [i64, i64, i64, d]
        lib._opim_ready = True
    return lib


def constants(n: int, k: int, eps: float, delta: float, cap: int = 0) -> dict:
    out = np.zeros(4, np.float64)
    _lib().orc_opim_constants(n, k, eps, delta, cap, out.ctypes.data)
    return dict(theta_max=out[0], theta0=int(out[1]), rounds=int(out[2]), a=out[3])


def lower(cov2: int, theta: int, n: int, a: float) -> float:
    return float(_lib().orc_opim_lower(cov2, theta, n, a))


def upper(cov1u: int, theta: int, n: int, a: float) -> float:
    return float(_lib().orc_opim_upper(cov1u, theta, n, a))


def sets_hit(pool, n: int, seeds) -> int:
    """Number of RRR sets of pool that contain at least one seed."""
    is_seed = np.zeros(n, bool)
    is_seed[np.asarray(seeds, np.int64)] = True
    hit = 0
    for i in range(pool.theta):
        if is_seed[pool.members[pool.set_off[i]:pool.set_off[i + 1]]].any():
            hit += 1
    return hit


def marginal_topk(pool, n: int, seeds, k: int) -> int:
    """Sum of the k largest marginal gains |S(v) \\ C(seeds)| over all v."""
    is_seed = np.zeros(n, bool)
    is_seed[np.asarray(seeds, np.int64)] = True
    cnt = np.zeros(n, np.int64)
    for i in range(pool.theta):
        mem = pool.members[pool.set_off[i]:pool.set_off[i + 1]]
        if not is_seed[mem].any():
            cnt[mem] += 1
    return int(np.sort(cnt)[::-1][:k].sum())


@dataclass
class OPIMResult:
    thetas: list
    cov1: list
    cov2: list
    cov1u: list
    alphas: list
    sigma_l: float
    sigma_u: float
    seeds: np.ndarray


def _select(n, pool, k, rg):
    inv = O.invert(n, pool)
    if rg is None:
        return O.greedy(n, pool, inv, k)
    P, pseed, trunc, bdelta = rg
    r = O.randgreedi(n, pool, inv, k, P, pseed, trunc, bdelta)
    return O.Cover(r.seeds, r.gains, r.coverage)


def _concat(parts):
    from .imm import _concat as cat
    return cat(parts)


def opim(graph, model: int, k: int, eps: float, delta: float, seed: int, cap: int = 0,
         randgreedi: tuple | None = None) -> OPIMResult:
    n = graph.n
    c = constants(n, k, eps, delta, cap)
    target = 1.0 - np.exp(-1.0) - eps
    r1, r2 = [], []
    have = 0
    res = OPIMResult([], [], [], [], [], 0.0, 0.0, np.zeros(0, np.int32))
    for i in range(1, c["rounds"] + 1):
        th = c["theta0"] << (i - 1)
        r1.append(O.sample(model, graph, seed, have, th - have))
        r2.append(O.sample(model, graph, seed, R2_FIRST + have, th - have))
        have = th
        p1, p2 = _concat(r1), _concat(r2)
        cover = _select(n, p1, k, randgreedi)
        cov2 = sets_hit(p2, n, cover.seeds)
        cov1u = cover.coverage + marginal_topk(p1, n, cover.seeds, k)
        sl = lower(cov2, th, n, c["a"])
        su = upper(cov1u, th, n, c["a"])
        res.thetas.append(th)
        res.cov1.append(cover.coverage)
        res.cov2.append(cov2)
        res.cov1u.append(cov1u)
        res.alphas.append(sl / su)
        res.sigma_l, res.sigma_u, res.seeds = sl, su, cover.seeds
        if sl / su >= target:
            break
    return res
