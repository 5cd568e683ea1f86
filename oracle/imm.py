"""IMM driver (Alg. 1) over the oracle's sampling and greedy -- TEST INFRASTRUCTURE ONLY.

Alg. 1 in the paper's order: Estimate (lambda', the doubling start), up to
floor(log2 n) - 1 martingale rounds that extend the same pool (sample ids keep
counting, Sec. 3.2), SelectSeeds, CheckGoodness; then theta = ceil(lambda*/LB)
fresh samples (ids after the rounds' ids) and a final SelectSeeds.  The
formulas of Estimate / CheckGoodness / f are not in the paper (it defers to
Tang et al. 2015 and Chen 2018); orc_imm_* in oracle.c writes them out.
The paper prints none of their values, so they are pinned from outside it
(tests/test_oracle_imm.py): lambda' and lambda* against values worked out
independently at the LiveJournal-shaped size; both against the failure
budgets they are derived from (Chernoff / martingale tails, with the exact
integer binomial); l' against the halved failure events; round counts and
round thetas in exact rational arithmetic; CheckGoodness by a hand-worked
case.  The tests also check the structure (doubling, stopping rule, final
count) and the guarantee the paper restates (seeds within 1 - 1/e - eps of
the optimum, exact on tiny graphs).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import oracle as O


def _imm_lib():
    lib = O._lib()
    if not hasattr(lib, "_imm_ready"):
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int32
        lib.orc_imm_constants.argtypes = [i64, i32, d, d, ctypes.c_void_p]
        lib.orc_imm_round_theta.restype = i64
        lib.orc_imm_round_theta.argtypes = [d, i64, i32]
        lib.orc_imm_check.restype = ctypes.c_int
        lib.orc_imm_check.argtypes = [i64, i64, i64, i32, d, ctypes.POINTER(d)]
        lib.orc_imm_final_theta.restype = i64
        lib.orc_imm_final_theta.argtypes = [d, d]
        lib._imm_ready = True
    return lib


def constants(n: int, k: int, eps: float, ell: float) -> dict:
    out = np.zeros(5, np.float64)
    _imm_lib().orc_imm_constants(n, k, eps, ell, out.ctypes.data)
    return dict(ell2=out[0], eps2=out[1], lambda_prime=out[2], lambda_star=out[3],
                rounds=int(out[4]))


@dataclass
class IMMResult:
    theta_rounds: list
    lb: float
    theta: int
    seeds: np.ndarray
    coverage: int


def _select(n, pool, k, rg):
    inv = O.invert(n, pool)
    if rg is None:
        return O.greedy(n, pool, inv, k)
    P, pseed, trunc, delta = rg
    r = O.randgreedi(n, pool, inv, k, P, pseed, trunc, delta)
    return O.Cover(r.seeds, r.gains, r.coverage)


def imm(graph, model: int, k: int, eps: float, ell: float, seed: int,
        randgreedi: tuple | None = None) -> IMMResult:
    """randgreedi = (P, partition seed, streamed seeds per part, delta) selects
    seeds with Alg. 4 + Alg. 5 in every round (GreediRIS); None: plain greedy."""
    lib = _imm_lib()
    n = graph.n
    c = constants(n, k, eps, ell)
    parts = []
    have = 0
    lb = 1.0
    thetas = []
    for i in range(1, c["rounds"] + 1):
        th = int(lib.orc_imm_round_theta(c["lambda_prime"], n, i))
        thetas.append(th)
        if th > have:                                   # Sample(G, theta_i - |R|, R)
            parts.append(O.sample(model, graph, seed, have, th - have))
            have = th
        pool = _concat(parts)
        cover = _select(n, pool, k, randgreedi)         # SelectSeeds
        lbv = ctypes.c_double()
        if lib.orc_imm_check(n, cover.coverage, th, i, c["eps2"], ctypes.byref(lbv)):
            lb = lbv.value
            break
    theta = int(lib.orc_imm_final_theta(c["lambda_star"], lb))
    final = O.sample(model, graph, seed, have, theta)   # fresh samples, ids after the rounds'
    cover = _select(n, final, k, randgreedi)
    return IMMResult(thetas, lb, theta, cover.seeds, cover.coverage)


def _concat(parts):
    set_off = [np.zeros(1, np.int64)]
    members = []
    base = 0
    ex = 0
    for p in parts:
        set_off.append(p.set_off[1:] + base)
        members.append(p.members)
        base += int(p.set_off[-1])
        ex += p.examined
    return O.Pool(np.concatenate(set_off), np.concatenate(members) if members else
                  np.zeros(0, np.int32), ex)
