"""Pins for the oracle's RRR sampling (Def. 3, Sec. 2.1 "Sample").

Each test checks the oracle against something other than itself: an explicit
live-edge world searched with scipy's BFS, exact inclusion probabilities from
enumerating every world (oracle/brute.py), or a closed-form special case.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order

from paper_2408_10982_gb300 import inputs

TWO32 = 1 << 32


def _reverse_reach_scipy(g, live, root):
    """Vertices with a live path to root: BFS from root on the reversed live graph."""
    dst = np.repeat(np.arange(g.n), np.diff(g.in_off))
    src = g.in_src.astype(np.int64)
    keep = live.astype(bool)
    # reversed edge dst -> src for every live edge src -> dst
    mat = sp.csr_matrix((np.ones(int(keep.sum())), (dst[keep], src[keep])), shape=(g.n, g.n))
    order = breadth_first_order(mat, root, directed=True, return_predecessors=False)
    return set(int(x) for x in order)


@pytest.mark.parametrize("wmode,gseed", [("random", 1), ("0.3", 2), ("0.05", 3), ("lt", 4)])
def test_ic_set_is_reverse_reachable_set_of_live_world(orc, wmode, gseed):
    g = inputs.random_graph(40, 200, gseed, wmode)
    seed = 1234 + gseed
    pool = orc.sample(orc.IC, g, seed, 0, 150)
    for s in range(150):
        live = np.array([orc.ic_coin(seed, s, e) < int(g.w[e]) for e in range(g.m)])
        root = orc.root(seed, s, g.n)
        want = _reverse_reach_scipy(g, live, root)
        got = pool.set(s)
        assert list(got) == sorted(want), s
        assert root in set(got.tolist())


def test_ic_set_ids_continue_across_calls(orc):
    """Sample ids are absolute: sets first..first+count-1 equal a slice of a longer run."""
    g = inputs.random_graph(30, 120, 9, "0.4")
    a = orc.sample(orc.IC, g, 5, 0, 60)
    b = orc.sample(orc.IC, g, 5, 25, 20)
    for j in range(20):
        assert np.array_equal(a.set(25 + j), b.set(j))


def _freq_check(orc, model, g, exact_fn, samples, seed):
    pool = orc.sample(model, g, seed, 0, samples)
    hits = np.zeros((g.n, g.n))
    roots = np.zeros(g.n)
    for s in range(samples):
        r = orc.root(seed, s, g.n)
        roots[r] += 1
        for v in pool.set(s):
            hits[r, v] += 1
    for r in range(g.n):
        p = np.array([float(x) for x in exact_fn(g, r)])
        f = hits[r] / roots[r]
        sigma = np.sqrt(np.maximum(p * (1 - p), 1e-12) / roots[r])
        assert np.all(np.abs(f - p) <= 5 * sigma + 1e-9), (r, f, p)


def test_ic_inclusion_probabilities_exact(orc):
    from oracle import brute
    g = inputs.random_graph(5, 9, 11, "random")
    _freq_check(orc, orc.IC, g, brute.ic_inclusion_exact, 100000, 77)


def test_lt_inclusion_probabilities_exact(orc):
    from oracle import brute
    g = inputs.random_graph(5, 10, 12, "lt_random")
    _freq_check(orc, orc.LT, g, brute.lt_inclusion_exact, 100000, 78)


def test_ic_special_cases(orc):
    g0 = inputs.random_graph(25, 120, 3, "zero")
    pool = orc.sample(orc.IC, g0, 9, 0, 100)
    for s in range(100):
        assert pool.set(s).tolist() == [orc.root(9, s, g0.n)]
    g1 = inputs.random_graph(25, 60, 4, "one")
    pool = orc.sample(orc.IC, g1, 9, 0, 100)
    everything_live = np.ones(g1.m)
    for s in range(100):
        r = orc.root(9, s, g1.n)
        assert pool.set(s).tolist() == sorted(_reverse_reach_scipy(g1, everything_live, r))


def _lt_pick(orc, g, seed, s, v):
    """The in-edge v keeps in world s: searchsorted over cumulative weights."""
    b, e = int(g.in_off[v]), int(g.in_off[v + 1])
    if e == b:
        return None
    cum = np.cumsum(g.w[b:e].astype(np.uint64))
    x = orc.lt_draw(seed, s, v)
    j = int(np.searchsorted(cum, np.uint64(x), side="right"))
    return None if j >= e - b else b + j


@pytest.mark.parametrize("wmode,gseed", [("lt", 21), ("lt_random", 22)])
def test_lt_set_is_backward_pick_chain(orc, wmode, gseed):
    g = inputs.random_graph(40, 220, gseed, wmode)
    seed = 99
    pool = orc.sample(orc.LT, g, seed, 0, 200, keep_order=True)
    for s in range(200):
        chain = [orc.root(seed, s, g.n)]
        while True:
            e = _lt_pick(orc, g, seed, s, chain[-1])
            if e is None:
                break
            u = int(g.in_src[e])
            if u in chain:
                break
            chain.append(u)
        assert pool.set(s).tolist() == chain, s
        # a simple path backwards along edges: consecutive entries are in-neighbours
        for a, b in zip(chain, chain[1:]):
            assert b in g.in_src[g.in_off[a]:g.in_off[a + 1]]
        assert len(set(chain)) == len(chain)


def test_lt_zero_weights_give_singletons(orc):
    g = inputs.random_graph(20, 80, 5, "zero")
    pool = orc.sample(orc.LT, g, 3, 0, 50)
    assert np.all(np.diff(pool.set_off) == 1)


def test_examined_counts(orc):
    """IC flips one coin per in-edge of every member; LT scans up to its pick."""
    g = inputs.random_graph(40, 200, 8, "0.2")
    pool = orc.sample(orc.IC, g, 4, 0, 80)
    indeg = np.diff(g.in_off)
    assert pool.examined == int(indeg[pool.members].sum())
    gl = inputs.random_graph(40, 200, 8, "lt")
    pool = orc.sample(orc.LT, gl, 4, 0, 80, keep_order=True)
    want = 0
    for s in range(80):
        for v in pool.set(s):
            e = _lt_pick(orc, gl, 4, s, int(v))
            want += (int(indeg[v]) if e is None else e - int(gl.in_off[v]) + 1)
    assert pool.examined == want


def test_rmat_fixture_shape():
    g = inputs.graph_small_ic()
    assert g.n == 1024 and g.m == 16384
    assert np.all(np.diff(g.in_off) >= 0) and g.in_off[-1] == g.m
    dst = np.repeat(np.arange(g.n), np.diff(g.in_off))
    assert np.all(g.in_src != dst)
    key = dst.astype(np.int64) * g.n + g.in_src
    assert np.all(np.diff(key) > 0)          # sorted by (dst, src), no repeats
    assert g.digest() == inputs.graph_small_ic().digest()
    assert np.all(g.w == inputs.quantise_probability(0.1)) and int(g.w[0]) == 429496730


def test_parallel_split_equals_one_call(orc):
    """The process-parallel oracle (id ranges split over spawned workers) gives
    exactly the single call's pool: sample ids key every draw."""
    from oracle import parallel
    g = inputs.rmat_graph(1 << 12, 1 << 16, 5, "lt")
    for model in (orc.IC, orc.LT):
        one = orc.sample(model, g, 11, 100, 5000)
        par = parallel.sample(model, g, 11, 100, 5000, workers=3, chunk=777)
        assert np.array_equal(one.set_off, par.set_off)
        assert np.array_equal(one.members, par.members)
        assert one.examined == par.examined
