"""Pins for the oracle's covering subsets, greedy, streaming and RandGreedi.

Checks against brute force on tiny instances (oracle/brute.py: from-scratch
marginal gains, optimal cover by enumeration), against the approximation
bounds the paper states (Sec. 3.2 (1-1/e); Lemma 2's truncated bound; Alg. 5's
threshold argument) and against the paper's printed numbers (63 buckets at
k = 100, delta = 0.077, Sec. 4.1; worst-case ratio 0.123 at eps = 0.13,
Sec. 4.2).
"""
import math

import numpy as np
import pytest

from oracle import brute
from paper_2408_10982_gb300 import inputs


def _instance(orc, n=12, m=40, theta=30, gseed=1, model=0, seed=5):
    g = inputs.random_graph(n, m, gseed, "0.35" if model == 0 else "lt")
    pool = orc.sample(model, g, seed, 0, theta)
    inv = orc.invert(g.n, pool)
    S = brute.covering_subsets(g.n, [pool.set(i) for i in range(theta)])
    return g, pool, inv, S


def test_invert_is_transpose(orc):
    g, pool, (vtx_off, set_ids), S = _instance(orc, n=30, m=150, theta=200)
    for v in range(g.n):
        assert set_ids[vtx_off[v]:vtx_off[v + 1]].tolist() == sorted(S[v])


@pytest.mark.parametrize("gseed", range(6))
@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_greedy_equals_from_scratch_definition(orc, gseed, k):
    g, pool, inv, S = _instance(orc, gseed=gseed, model=gseed % 2)
    c = orc.greedy(g.n, pool, inv, k)
    seeds, gains, cov = brute.greedy_definition(S, k)
    assert c.seeds.tolist() == seeds
    assert c.gains.tolist() == gains
    assert c.coverage == cov == brute.coverage(S, seeds)
    # restricted candidate list (a partition's local greedy)
    cand = [v for v in range(g.n) if (v * 7 + gseed) % 3 == 0]
    c2 = orc.greedy(g.n, pool, inv, k, np.array(cand, dtype=np.int32))
    s2, g2, cov2 = brute.greedy_definition(S, k, cand)
    assert c2.seeds.tolist() == s2 and c2.gains.tolist() == g2 and c2.coverage == cov2


@pytest.mark.parametrize("gseed", range(8))
def test_greedy_approximation_and_truncation_bounds(orc, gseed):
    """Greedy's first j picks cover >= (1-(1-1/k)^j) OPT_k (proof of Lemma 2);
    j = k gives the classic (1-(1-1/k)^k) >= 1-1/e of Sec. 3.2."""
    g, pool, inv, S = _instance(orc, n=11, m=45, theta=40, gseed=gseed + 10)
    for k in (2, 3, 4):
        c = orc.greedy(g.n, pool, inv, k)
        opt = brute.optimal_cover(S, k)
        for j in range(1, k + 1):
            assert c.gains[:j].sum() >= (1 - (1 - 1 / k) ** j) * opt - 1e-9
        assert c.coverage >= (1 - 1 / math.e) * opt - 1e-9


def test_greedy_invariants_on_rmat(orc):
    g = inputs.graph_small_ic()
    pool = orc.sample(orc.IC, g, 42, 0, 4000)
    inv = orc.invert(g.n, pool)
    c = orc.greedy(g.n, pool, inv, 16)
    assert len(set(c.seeds.tolist())) == len(c.seeds)
    assert np.all(np.diff(c.gains) <= 0)           # submodularity: gains never grow
    vtx_off, set_ids = inv
    union = set()
    for v in c.seeds:
        union |= set(set_ids[vtx_off[v]:vtx_off[v + 1]].tolist())
    assert c.coverage == int(c.gains.sum()) == len(union)
    assert int(c.gains[0]) == int(np.diff(vtx_off).max())


def test_greedy_tie_break_and_zero_gain(orc):
    # sets: R0={1,3}, R1={3,5}, R2={1,5}; |S(1)|=|S(3)|=|S(5)|=2 -> smallest id first
    class P:  # a hand-made pool
        set_off = np.array([0, 2, 4, 6], dtype=np.int64)
        members = np.array([1, 3, 3, 5, 1, 5], dtype=np.int32)
        theta = 3
    inv = orc.invert(6, P)
    c = orc.greedy(6, P, inv, 5)
    # S(1)={0,2}, S(3)={0,1}, S(5)={1,2}: pick 1 (tie of three, smallest id),
    # then S(3) and S(5) both gain {1}: pick 3; then every gain is zero: stop.
    assert c.seeds.tolist() == [1, 3] and c.gains.tolist() == [2, 1] and c.coverage == 3
    seeds, gains, cov = brute.greedy_definition(
        brute.covering_subsets(6, [[1, 3], [3, 5], [1, 5]]), 5)
    assert c.seeds.tolist() == seeds and c.gains.tolist() == gains and c.coverage == cov


def test_bucket_count_matches_paper(orc):
    # Sec. 4.1: delta = 0.077 gives 63 buckets at k = 100.
    assert orc.num_buckets(100, 0.077) == 63
    for k, d in [(100, 0.077), (16, 0.1), (1000, 0.0562), (2, 0.3), (1, 0.2)]:
        B = orc.num_buckets(k, d)
        assert B >= 1
        if k > 1:
            assert (1 + d) ** (B - 1) < k <= (1 + d) ** B * (1 + 1e-12)


def test_streaming_ratio_matches_paper(orc):
    # Sec. 4.2: eps = 0.13, delta = 0.077 give a worst-case ratio of 0.123.
    assert round(orc.ratio_streaming(0.13, 0.077), 3) == 0.123
    # Lemma 3 at alpha = 1 has the same form as Lemma 1
    assert orc.ratio_truncated_streaming(1.0, 0.13, 0.077) == pytest.approx(
        orc.ratio_streaming(0.13, 0.077))


def test_bucket_thresholds(orc):
    for l, k, d in [(7296, 16, 0.077), (1000, 100, 0.077), (5, 3, 0.2), (123456, 200, 0.05)]:
        thr = orc.bucket_thresholds(l, k, d)
        for b, t in enumerate(thr):
            exact = l * (1 + d) ** b / (2 * k)
            assert t == math.ceil(exact) or abs(exact - round(exact)) < 1e-6


@pytest.mark.parametrize("gseed", range(10))
def test_stream_buckets_half_opt_bound(orc, gseed):
    """Alg. 5's argument: for the bucket whose guess v_b lies in (OPT/(1+d), OPT],
    either k seeds each gained >= v_b/(2k), or every rejected optimal subset
    gained < v_b/(2k); both give |C_b| >= v_b/2 >= OPT/(2(1+d))."""
    g, pool, inv, S = _instance(orc, n=12, m=50, theta=45, gseed=gseed + 30)
    rng = np.random.default_rng(gseed)
    stream = rng.permutation(g.n)[: 9]
    k, d = 3, 0.2
    l = max(len(S[v]) for v in stream)
    if l == 0:
        pytest.skip("empty stream")
    thr = orc.bucket_thresholds(l, k, d)
    bk = orc.stream_buckets(pool.theta, inv, stream, k, thr)
    opt = brute.optimal_cover(S, k, cand=stream)
    assert bk.cov.max() >= opt / (2 * (1 + d)) - 1e-9
    # each bucket's coverage is the union of its seeds, gains as recorded
    for b in range(thr.size):
        seeds = bk.seeds[b, : bk.n[b]].tolist()
        assert brute.coverage(S, seeds) == bk.cov[b] == bk.gains[b, : bk.n[b]].sum()
        assert bk.n[b] <= k


def test_stream_single_bucket_is_threshold_streaming(orc):
    """B = 1 reduces to the textbook one-threshold rule: accept while < k and gain >= T."""
    g, pool, inv, S = _instance(orc, n=14, m=60, theta=50, gseed=3)
    stream = list(range(g.n))
    k, T = 4, 3
    bk = orc.stream_buckets(pool.theta, inv, stream, k, np.array([T], dtype=np.int64))
    covered, picked = set(), []
    for x in stream:
        if len(picked) < k and len(S[x] - covered) >= T:
            picked.append(x)
            covered |= S[x]
    assert bk.seeds[0, : bk.n[0]].tolist() == picked and bk.cov[0] == len(covered)


@pytest.mark.parametrize("gseed", range(5))
@pytest.mark.parametrize("P,trunc", [(3, 1), (4, 2), (2, 3)])
def test_randgreedi(orc, gseed, P, trunc):
    g, pool, inv, S = _instance(orc, n=16, m=70, theta=60, gseed=gseed + 50, model=gseed % 2)
    k, d, pseed = 3, 0.1, 17 + gseed
    rg = orc.randgreedi(g.n, pool, inv, k, P, pseed, trunc, d)
    part = orc.partition(g.n, P, pseed)
    # Alg. 4: local greedy of partition p over its own covering subsets
    for p in range(P):
        cand = [v for v in range(g.n) if part[v] == p]
        seeds, gains, cov = brute.greedy_definition(S, k, cand)
        assert rg.local_seeds[p, : rg.local_n[p]].tolist() == seeds
        assert rg.local_gains[p, : rg.local_n[p]].tolist() == gains
        assert rg.local_cov[p] == cov
    # stream order (rank j, then partition p), first `trunc` seeds of each partition
    stream = [int(rg.local_seeds[p, j]) for j in range(min(trunc, k)) for p in range(P)
              if j < rg.local_n[p]]
    l = int(np.diff(inv[0]).max())
    bk = orc.stream_buckets(pool.theta, inv, stream, k, orc.bucket_thresholds(l, k, d))
    assert np.array_equal(bk.cov, rg.buckets.cov) and np.array_equal(bk.seeds, rg.buckets.seeds)
    # Alg. 4: the better of the best bucket and the best local solution
    assert rg.coverage == max(int(rg.buckets.cov.max()), int(rg.local_cov.max()))
    assert rg.coverage == brute.coverage(S, rg.seeds.tolist())
    if rg.chosen == -1:
        assert rg.buckets.cov.max() >= rg.local_cov.max()
    else:
        assert rg.local_cov[rg.chosen] > rg.buckets.cov.max()
        assert rg.chosen == int(np.argmax(rg.local_cov))
    assert len(rg.seeds) <= k


def test_trunc_count():
    from oracle import trunc_count
    assert trunc_count(100, 1, 4) == 25
    assert trunc_count(100, 1, 8) == 13       # ceil(12.5)
    assert trunc_count(5, 1, 100) == 1
    assert trunc_count(7, 1, 1) == 7


# ---------------------------------------------------------------------------
# Lazy greedy (Alg. 2) and Alg. 4's non-streaming global step
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("gseed", range(8))
@pytest.mark.parametrize("k", [1, 3, 6, 40])
def test_lazy_greedy_equals_from_scratch_definition(orc, gseed, k):
    """Stale gains are upper bounds (submodularity), so Alg. 2 with the key
    order (gain, smaller id) picks what the standard greedy picks; also with a
    candidate list, and past the point where every gain is zero."""
    g, pool, inv, S = _instance(orc, gseed=gseed + 70, model=gseed % 2)
    c = orc.lazy_greedy(g.n, pool, inv, k)
    seeds, gains, cov = brute.greedy_definition(S, k)
    assert c.seeds.tolist() == seeds and c.gains.tolist() == gains and c.coverage == cov
    cand = [v for v in range(g.n) if (v * 5 + gseed) % 3 != 0]
    c2 = orc.lazy_greedy(g.n, pool, inv, k, np.array(cand, dtype=np.int32))
    s2, g2, cov2 = brute.greedy_definition(S, k, cand)
    assert c2.seeds.tolist() == s2 and c2.gains.tolist() == g2 and c2.coverage == cov2


@pytest.mark.parametrize("theta", [3, 40, 5000])
def test_lazy_greedy_equals_standard_greedy_on_rmat(orc, theta):
    """Tie-heavy (theta = 3: almost every gain is 1) to many sets."""
    g = inputs.rmat_graph(1 << 12, 1 << 16, 3, "lt")
    pool = orc.sample(orc.LT, g, 9, 0, theta)
    inv = orc.invert(g.n, pool)
    for k in (1, 10, 100):
        a, b = orc.greedy(g.n, pool, inv, k), orc.lazy_greedy(g.n, pool, inv, k)
        assert a.seeds.tolist() == b.seeds.tolist() and a.gains.tolist() == b.gains.tolist()
        assert a.coverage == b.coverage


def test_lazy_greedy_hand_worked():
    """Alg. 2 step by step on R0 = {0, 1}, R1 = {1, 2}, R2 = {2}, R3 = {0, 3}:
    S(0) = {0, 3}, S(1) = {0, 1}, S(2) = {1, 2}, S(3) = {3}.  Heap keys 2, 2, 2, 1.
    Pop 0 (ties: smallest id), gain 2 >= top key 2 (vertex 1, larger id): take 0.
    Pop 1, gain |{0,1} - {0,3}| = 1 < top key 2 (vertex 2): push (1, 1).
    Pop 2, gain 2 >= top 1: take 2.  Pop 1, gain 0 < top key 1 (vertex 3):
    push (1, 0).  Pop 3, gain 0; the top (vertex 1, key 0) ranks above it: push
    (3, 0).  Pop 1, gain 0, ranks above the top (3, 0): it would be taken with
    gain 0, so the selection stops.  Seeds [0, 2], gains [2, 2]."""
    import oracle
    oracle.build()

    class P:
        set_off = np.array([0, 2, 4, 5, 7], dtype=np.int64)
        members = np.array([0, 1, 1, 2, 2, 0, 3], dtype=np.int32)
        theta = 4
    inv = oracle.invert(4, P)
    c = oracle.lazy_greedy(4, P, inv, 4)
    assert c.seeds.tolist() == [0, 2] and c.gains.tolist() == [2, 2] and c.coverage == 4


@pytest.mark.parametrize("gseed", range(5))
@pytest.mark.parametrize("P,trunc", [(3, 1), (4, 2), (2, 3)])
def test_randgreedi_naive_global_step(orc, gseed, P, trunc):
    """Alg. 4 as written: the global solution is the greedy over the union of
    the gathered local seeds (the first `trunc` of every part); the answer is
    the better of it and the best local solution (ties: the global one)."""
    g, pool, inv, S = _instance(orc, n=16, m=70, theta=60, gseed=gseed + 90, model=gseed % 2)
    k, pseed = 3, 23 + gseed
    rg = orc.randgreedi(g.n, pool, inv, k, P, pseed, trunc, 0.1, naive=True)
    ref = orc.randgreedi(g.n, pool, inv, k, P, pseed, trunc, 0.1)
    assert np.array_equal(rg.local_seeds, ref.local_seeds)
    assert np.array_equal(rg.local_cov, ref.local_cov)
    gathered = sorted(int(rg.local_seeds[p, j]) for p in range(P)
                      for j in range(min(trunc, int(rg.local_n[p]))))
    seeds, gains, cov = brute.greedy_definition(S, k, gathered)
    assert rg.buckets.n.tolist() == [len(seeds)] and rg.thr.tolist() == [0]
    assert rg.buckets.seeds[0, : len(seeds)].tolist() == seeds
    assert rg.buckets.gains[0, : len(seeds)].tolist() == gains
    assert int(rg.buckets.cov[0]) == cov
    assert rg.coverage == max(cov, int(rg.local_cov.max()))
    assert rg.coverage == brute.coverage(S, rg.seeds.tolist())
    assert (rg.chosen == -1) == (cov >= int(rg.local_cov.max()))
