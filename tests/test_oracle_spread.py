"""Pins for the oracle's forward simulation (the spread sigma(S) of a seed set).

Run r simulates the live-edge world of RRR sample r, so by the RIS identity
the root of sample r is activated from S exactly when S meets RRR set r: the
forward BFS over out-edges and the reverse BFS / backward walk over in-edges
are independent computations of the same world and must agree run by run.
The mean over runs is pinned to sigma(S) computed exactly by enumerating
every live-edge world of tiny graphs.
"""
import numpy as np
import pytest

from paper_2408_10982_gb300 import inputs


def _hits_from_pool(pool, seeds):
    s = set(int(x) for x in seeds)
    return np.array([1 if s & set(int(v) for v in pool.set(i)) else 0
                     for i in range(pool.theta)], np.uint8)


@pytest.mark.parametrize("model,wmode", [(0, "random"), (0, "0.2"), (1, "lt"), (1, "lt_random")])
@pytest.mark.parametrize("gseed", [3, 4])
def test_root_hit_equals_rrr_intersection(orc, model, wmode, gseed):
    g = inputs.random_graph(40, 160, gseed, wmode)
    rng = np.random.default_rng(gseed)
    for size in (1, 2, 5):
        seeds = rng.choice(g.n, size=size, replace=False)
        act, hit = orc.spread(model, g, 17, 100, 400, seeds)
        pool = orc.sample(model, g, 17, 100, 400)
        assert np.array_equal(hit, _hits_from_pool(pool, seeds))
        assert np.all(act >= size)


def test_root_hit_identity_on_rmat(orc):
    for model, w in ((0, "ic0.1"), (1, "lt")):
        g = inputs.rmat_graph(1 << 12, 1 << 16, 5, w)
        seeds = np.array([0, 1, 2, 512, 4095])
        act, hit = orc.spread(model, g, 42, 0, 3000, seeds)
        pool = orc.sample(model, g, 42, 0, 3000)
        assert np.array_equal(hit, _hits_from_pool(pool, seeds))


@pytest.mark.parametrize("model,wmode,gseed", [(0, "random", 21), (1, "lt_random", 22)])
def test_mean_matches_exact_spread(orc, model, wmode, gseed):
    from oracle import brute
    g = inputs.random_graph(5, 9 if model == 0 else 10, gseed, wmode)
    seeds = [0, 3]
    exact = float(brute.ic_spread_exact(g, seeds) if model == 0 else brute.lt_spread_exact(g, seeds))
    runs = 100000
    act, hit = orc.spread(model, g, 99, 0, runs, seeds)
    sd = act.std() / np.sqrt(runs)
    assert abs(act.mean() - exact) <= 5 * sd + 1e-9
    # the RIS estimator n * P(root activated) has the same expectation
    sd2 = g.n * hit.std() / np.sqrt(runs)
    assert abs(g.n * hit.mean() - exact) <= 5 * sd2 + 1e-9


def test_special_cases(orc):
    g0 = inputs.random_graph(25, 120, 3, "zero")
    act, _ = orc.spread(0, g0, 1, 0, 50, [4, 4, 7])
    assert np.all(act == 2)                       # nothing is live: only the distinct seeds
    g1 = inputs.random_graph(25, 120, 3, "one")   # every edge (almost surely) live
    act, _ = orc.spread(0, g1, 1, 0, 50, [4])
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    n = g1.n
    dst = np.repeat(np.arange(n), np.diff(g1.in_off))
    adj = sp.csr_matrix((np.ones(g1.m), (g1.in_src, dst)), shape=(n, n))
    reach = breadth_first_order(adj, 4, directed=True, return_predecessors=False)
    assert np.all(act == len(reach))


@pytest.mark.parametrize("model,wmode,gseed", [(0, "random", 31), (0, "0.3", 32),
                                               (1, "lt_random", 33), (1, "lt", 34)])
def test_ris_identity_exact_between_the_brute_forces(model, wmode, gseed):
    """The identity RIS rests on (Def. 3, Sec. 2.1): sigma(S) = n P[S meets
    RRR(r)] for a uniform root r; for one seed v, sigma({v}) = sum over roots
    r of P[v in RRR(r)].  Forward reach over every live-edge world and reverse
    reach (IC) / the backward pick chain (LT) from every root are independent
    brute-force computations; they must agree exactly, as rationals."""
    from oracle import brute
    g = inputs.random_graph(5, 8, gseed, wmode)
    incl = brute.ic_inclusion_exact if model == 0 else brute.lt_inclusion_exact
    spread = brute.ic_spread_exact if model == 0 else brute.lt_spread_exact
    per_root = [incl(g, r) for r in range(g.n)]
    for v in range(g.n):
        assert sum(pr[v] for pr in per_root) == spread(g, [v])
