"""GPU path (through the C ABI) against the CPU oracle, element by element.

RRR sets, covering subsets, partitions, seeds, gains and coverage are integer
results: the bar is bit-exact equality.  Set ids inside one S(v) are compared
as sorted lists (their order is unspecified).
"""
import numpy as np
import pytest

import oracle as O
from paper_2408_10982_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def im():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_10982_gb300 import build, im as imm
    build.build_library()
    O.build()
    return imm


def gpu_pool(im, g, model, seed, ids, cap_entries=None):
    G = im.Graph(g)
    theta = sum(c for _, c in ids)
    cap = cap_entries if cap_entries is not None else max(1, theta) * g.n
    P = im.Pool(G, max(theta, 1), min(cap, 1 << 31))
    for first, count in ids:
        P.sample(model, seed, first, count)
    return G, P


def oracle_pool(g, model, seed, ids):
    parts = [O.sample(model, g, seed, f, c) for f, c in ids]
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


def assert_pool_equal(im, P, ref):
    set_off, members = P.export()
    assert set_off.shape == ref.set_off.shape
    assert np.array_equal(set_off, ref.set_off)
    assert np.array_equal(members, ref.members)
    theta, total, examined = P.info()
    assert examined == ref.examined


def assert_index_equal(P, g, ref):
    vtx_off, set_ids = P.index()
    rv, rs = O.invert(g.n, ref)
    assert np.array_equal(vtx_off, rv)
    for v in range(g.n):
        a, b = vtx_off[v], vtx_off[v + 1]
        if b - a > 1:
            assert np.array_equal(np.sort(set_ids[a:b]), rs[a:b]), v
        elif b - a == 1:
            assert set_ids[a] == rs[a]


# --- sampling ---------------------------------------------------------------

def test_ic_small_rmat_full(im):
    """R-MAT scale 10, IC p = 0.1, 16,384 sets: the whole pool bit-exact."""
    g = inputs.graph_small_ic()
    G, P = gpu_pool(im, g, im.IM_IC, 42, [(0, 16384)])
    ref = O.sample(O.IC, g, 42, 0, 16384)
    assert_pool_equal(im, P, ref)
    assert_index_equal(P, g, ref)
    c = P.cover(16)
    rc = O.greedy(g.n, ref, O.invert(g.n, ref), 16)
    assert c.seeds.tolist() == rc.seeds.tolist()
    assert c.gains.tolist() == rc.gains.tolist()
    assert c.coverage == rc.coverage


@pytest.mark.parametrize("wmode", ["random", "0.3", "0.05", "zero", "one", "lt"])
@pytest.mark.parametrize("theta", [1, 31, 33, 1000])
def test_ic_random_graphs(im, wmode, theta):
    g = inputs.random_graph(60, 400, 7, wmode)
    G, P = gpu_pool(im, g, im.IM_IC, 1234, [(0, theta)])
    assert_pool_equal(im, P, O.sample(O.IC, g, 1234, 0, theta))


@pytest.mark.parametrize("wmode", ["lt", "lt_random", "zero"])
@pytest.mark.parametrize("theta", [1, 33, 2000])
def test_lt_random_graphs(im, wmode, theta):
    g = inputs.random_graph(60, 500, 9, wmode)
    G, P = gpu_pool(im, g, im.IM_LT, 99, [(0, theta)])
    assert_pool_equal(im, P, O.sample(O.LT, g, 99, 0, theta))


def test_lt_rmat_scale14(im):
    g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
    G, P = gpu_pool(im, g, im.IM_LT, 42, [(0, 50000)])
    ref = O.sample(O.LT, g, 42, 0, 50000)
    assert_pool_equal(im, P, ref)
    assert_index_equal(P, g, ref)


def test_ic_rmat_global_visited(im):
    """n > 65,536 puts the visited bitmaps in global memory."""
    g = inputs.rmat_graph(1 << 17, 1 << 21, 42, "trivalency")
    G, P = gpu_pool(im, g, im.IM_IC, 5, [(0, 20000)])
    assert_pool_equal(im, P, O.sample(O.IC, g, 5, 0, 20000))


def test_ic_giant_sets_overflow_path(im):
    """Sets larger than a warp's queue (16,384) and than a block sort (16,384)."""
    g = inputs.rmat_graph(1 << 15, 1 << 19, 3, "ic0.9")
    G, P = gpu_pool(im, g, im.IM_IC, 8, [(0, 300)], cap_entries=300 * (1 << 15))
    ref = O.sample(O.IC, g, 8, 0, 300)
    assert np.diff(ref.set_off).max() > 16384
    assert_pool_equal(im, P, ref)


def test_append_matches_one_call(im):
    g = inputs.random_graph(50, 300, 4, "0.25")
    G, P = gpu_pool(im, g, im.IM_IC, 77, [(0, 100), (100, 37), (137, 500)])
    assert_pool_equal(im, P, O.sample(O.IC, g, 77, 0, 637))
    G2, P2 = gpu_pool(im, g, im.IM_IC, 77, [(1000, 200), (5, 10)])
    assert_pool_equal(im, P2, oracle_pool(g, O.IC, 77, [(1000, 200), (5, 10)]))


def test_capacity_error_leaves_pool_unchanged(im):
    g = inputs.random_graph(50, 300, 4, "one")
    G = im.Graph(g)
    P = im.Pool(G, 100, 120)
    with pytest.raises(im.ImError) as e:
        P.sample(im.IM_IC, 1, 0, 100)
    assert e.value.status == im.IM_ERR_CAPACITY
    assert P.info()[:2] == (0, 0)
    P2 = im.Pool(G, 10, 10 * 50)
    with pytest.raises(im.ImError):
        P2.sample(im.IM_IC, 1, 0, 11)


def test_invalid_graph_rejected(im):
    g = inputs.random_graph(20, 50, 4, "0.5")
    bad = g.in_src.copy()
    bad[3] = 99
    with pytest.raises(im.ImError) as e:
        im.im_graph_create(g.in_off, bad, g.w, g.n, g.m)
    assert e.value.status == im.IM_ERR_INVALID_ARG


# --- partition and covers ---------------------------------------------------

def test_partition_labels(im):
    part = np.zeros(100000, np.int32)
    im.im_partition(100000, 148, 42, part)
    assert np.array_equal(part, O.partition(100000, 148, 42))


@pytest.mark.parametrize("k", [1, 3, 16, 64])
def test_greedy_plain(im, k):
    g = inputs.rmat_graph(4096, 65536, 11, "ic0.05")
    G, P = gpu_pool(im, g, im.IM_IC, 3, [(0, 20000)])
    ref = O.sample(O.IC, g, 3, 0, 20000)
    c = P.cover(k)
    rc = O.greedy(g.n, ref, O.invert(g.n, ref), k)
    assert c.seeds.tolist() == rc.seeds.tolist()
    assert c.gains.tolist() == rc.gains.tolist()
    assert c.coverage == rc.coverage


def test_greedy_stops_at_zero_gain(im):
    g = inputs.random_graph(30, 60, 2, "zero")      # every set is a singleton
    G, P = gpu_pool(im, g, im.IM_IC, 3, [(0, 10)])
    ref = O.sample(O.IC, g, 3, 0, 10)
    c = P.cover(25)
    rc = O.greedy(g.n, ref, O.invert(g.n, ref), 25)
    assert len(c.seeds) == len(rc.seeds) < 25
    assert c.seeds.tolist() == rc.seeds.tolist()
    assert c.coverage == rc.coverage == 10


def test_empty_pool_cover(im):
    g = inputs.random_graph(30, 60, 2, "0.5")
    G = im.Graph(g)
    P = im.Pool(G, 10, 100)
    c = P.cover(5)
    assert len(c.seeds) == 0 and c.coverage == 0


def _rg_compare(im, g, model, theta, k, Pn, alpha, delta, fused, seed=42, pseed=42,
                naive=False):
    G, P = gpu_pool(im, g, model, seed, [(0, theta)])
    ref = O.sample(model, g, seed, 0, theta)
    inv = O.invert(g.n, ref)
    trunc = O.trunc_count(k, *alpha)
    r = O.randgreedi(g.n, ref, inv, k, Pn, pseed, trunc, delta, naive=naive)
    opts = im.cover_opts(im.IM_RANDGREEDI, Pn, alpha, delta, pseed, fused,
                         im.IM_AGG_GREEDY if naive else im.IM_AGG_STREAM)
    c = P.cover(k, opts)
    B = 1 if naive else O.num_buckets(k, delta)
    d = P.randgreedi_details(k, Pn, B)
    assert np.array_equal(d["local_n"], r.local_n)
    for p in range(Pn):
        n_p = r.local_n[p]
        assert d["local_seeds"][p, :n_p].tolist() == r.local_seeds[p, :n_p].tolist(), p
        assert d["local_gains"][p, :n_p].tolist() == r.local_gains[p, :n_p].tolist(), p
    assert np.array_equal(d["local_cov"], r.local_cov)
    assert np.array_equal(d["thr"], r.thr)
    assert np.array_equal(d["bucket_n"], r.buckets.n)
    assert np.array_equal(d["bucket_cov"], r.buckets.cov)
    for b in range(B):
        nb = r.buckets.n[b]
        assert d["bucket_seeds"][b, :nb].tolist() == r.buckets.seeds[b, :nb].tolist(), b
        assert d["bucket_gains"][b, :nb].tolist() == r.buckets.gains[b, :nb].tolist(), b
    assert d["chosen"] == r.chosen
    assert c.seeds.tolist() == r.seeds.tolist()
    assert c.gains.tolist() == r.gains.tolist()
    assert c.coverage == r.coverage


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("Pn,alpha", [(148, (1, 4)), (7, (1, 1)), (1, (1, 2))])
def test_randgreedi_lt(im, fused, Pn, alpha):
    g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
    _rg_compare(im, g, im.IM_LT, 30000, 100 if Pn == 148 else 20, Pn, alpha, 0.077, fused)


@pytest.mark.parametrize("fused", [True, False])
def test_randgreedi_ic_small(im, fused):
    g = inputs.graph_small_ic()
    _rg_compare(im, g, im.IM_IC, 16384, 16, 148, (1, 4), 0.077, fused)


@pytest.mark.parametrize("group", [1, 8, 16, 32])
def test_lt_group_sizes_identical(im, group):
    """Lanes per LT walk is a tuning knob: every setting gives the same pool."""
    g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
    old = im.im_tune_get(im.IM_TUNE_LT_GROUP)
    im.im_tune_set(im.IM_TUNE_LT_GROUP, group)
    try:
        G, P = gpu_pool(im, g, im.IM_LT, 7, [(0, 20000)])
        assert_pool_equal(im, P, O.sample(O.LT, g, 7, 0, 20000))
        gr = inputs.random_graph(60, 500, 9, "lt_random")
        G2, P2 = gpu_pool(im, gr, im.IM_LT, 99, [(0, 999)])
        assert_pool_equal(im, P2, O.sample(O.LT, gr, 99, 0, 999))
    finally:
        im.im_tune_set(im.IM_TUNE_LT_GROUP, old)


@pytest.mark.parametrize("cache", [0, 1, 2])
def test_lt_cache_policies_identical(im, cache):
    """The L2 policy of the LT walk's loads changes no set."""
    g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
    ref = O.sample(O.LT, g, 5, 0, 40000)
    im.im_tune_set(im.IM_TUNE_LT_CACHE, cache)
    try:
        G, P = gpu_pool(im, g, im.IM_LT, 5, [(0, 40000)], cap_entries=40000 * 512)
        assert_pool_equal(im, P, ref)
    finally:
        im.im_tune_set(im.IM_TUNE_LT_CACHE, 0)


@pytest.mark.parametrize("cluster", [-1, 1, 2, 4, 8])
def test_randgreedi_bucket_stage_variants(im, cluster):
    """Two-launch RandGreedi: every bucket-stage layout (global bitmaps, or a
    shared-memory bitmap split over 1..8 blocks of a cluster) gives the oracle's result."""
    old = im.im_tune_get(im.IM_TUNE_RG_CLUSTER)
    im.im_tune_set(im.IM_TUNE_RG_CLUSTER, cluster)
    try:
        g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
        _rg_compare(im, g, im.IM_LT, 30000, 50, 148, (1, 4), 0.077, False)
    finally:
        im.im_tune_set(im.IM_TUNE_RG_CLUSTER, old)


@pytest.mark.parametrize("cluster", [0, -1])
def test_randgreedi_fused_layouts(im, cluster):
    """One-launch RandGreedi (producers and bucket consumers in one cooperative
    launch, the consumers reading slots as they are published) under both
    bucket-stage knob values gives the oracle's result, with 148 and with 100
    parts."""
    old = im.im_tune_get(im.IM_TUNE_RG_CLUSTER)
    im.im_tune_set(im.IM_TUNE_RG_CLUSTER, cluster)
    try:
        g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
        _rg_compare(im, g, im.IM_LT, 30000, 50, 148, (1, 4), 0.077, True)
        _rg_compare(im, g, im.IM_LT, 30000, 50, 100, (1, 8), 0.077, True)
    finally:
        im.im_tune_set(im.IM_TUNE_RG_CLUSTER, old)


def test_randgreedi_large_theta_cluster(im):
    """theta above one block's shared memory: the automatic cluster has >= 2 blocks."""
    g = inputs.rmat_graph(1 << 12, 1 << 16, 5, "lt")
    _rg_compare(im, g, im.IM_LT, 2_000_000, 40, 148, (1, 4), 0.077, False, seed=3)


@pytest.mark.parametrize("model,wts,rg", [("ic", "trivalency", False), ("lt", "lt", False),
                                          ("ic", "ic0.05", True)])
def test_imm_solve_matches_oracle(im, model, wts, rg):
    """im_solve (Alg. 1 on the device path) against the oracle's IMM driver:
    the same theta of every round, LB, final theta, seeds and coverage."""
    from oracle import imm as OI
    g = inputs.rmat_graph(4096, 65536, 7, wts)
    m = im.IM_IC if model == "ic" else im.IM_LT
    k, eps = 10, 0.5
    opts = im.cover_opts(im.IM_RANDGREEDI, 16, (1, 2), 0.1, 9, False) if rg else None
    ref = OI.imm(g, O.IC if model == "ic" else O.LT, k, eps, 1.0, 42,
                 randgreedi=(16, 9, O.trunc_count(k, 1, 2), 0.1) if rg else None)
    G = im.Graph(g)
    seeds, cov, theta, info = im.im_solve(G.handle, m, k, eps, 1.0, 42, opts)
    assert list(info.theta_rounds[: info.rounds]) == ref.theta_rounds
    assert info.lb == ref.lb
    assert theta == ref.theta == info.theta
    assert seeds.tolist() == ref.seeds.tolist()
    assert cov == ref.coverage


def test_solve_batch_matches_oracle_and_single_path(im):
    """A mixed batch (graphs of several sizes, IC and LT, uneven k and theta):
    every query gets the oracle's seeds, gains and coverage -- the same as alone."""
    graphs = {
        "a": inputs.rmat_graph(1 << 12, 1 << 16, 1, "ic0.1"),
        "b": inputs.rmat_graph(1 << 13, 1 << 17, 2, "lt"),
        "c": inputs.random_graph(50, 300, 3, "0.3"),
        "d": inputs.rmat_graph(1 << 17, 1 << 21, 4, "lt"),
    }
    G = {k: im.Graph(g) for k, g in graphs.items()}
    rng = np.random.default_rng(0)
    queries = []
    for q in range(23):
        name = "abcd"[q % 4]
        g = graphs[name]
        model = im.IM_LT if name in "bd" else im.IM_IC
        k = int(rng.integers(1, min(40, g.n) + 1))
        theta = int(rng.integers(0, 6000)) if q % 5 else 1
        queries.append((name, model, k, theta, int(rng.integers(0, 2**62))))
    batch = im.im_batch_create()
    try:
        for _ in range(2):                    # the arenas are reused on the second call
            out = im.im_solve_batch(batch, [(G[n].handle, m, k, th, sd)
                                            for n, m, k, th, sd in queries], 40)
            for (name, m, k, th, sd), (seeds, gains, cov, entries) in zip(queries, out):
                g = graphs[name]
                pool = O.sample(O.IC if m == im.IM_IC else O.LT, g, sd, 0, th)
                rc = O.greedy(g.n, pool, O.invert(g.n, pool), k)
                assert seeds.tolist() == rc.seeds.tolist(), (name, k, th)
                assert gains.tolist() == rc.gains.tolist()
                assert cov == rc.coverage and entries == pool.members.size
    finally:
        im.im_batch_destroy(batch)


def test_solve_batch_randgreedi_queries(im):
    """Batched RandGreedi queries (plain greedy ones beside them): a fixed
    partition count, and an open one the batch picks by timing -- every query
    equals the oracle's RandGreedi with the count the batch reports, and the
    same query alone through im_max_k_cover."""
    graphs = {"a": inputs.rmat_graph(1 << 12, 1 << 16, 1, "lt"),
              "b": inputs.rmat_graph(1 << 13, 1 << 17, 2, "ic0.05"),
              "c": inputs.rmat_graph(1 << 14, 1 << 18, 3, "lt")}
    G = {k: im.Graph(g) for k, g in graphs.items()}
    rg = lambda P, a: im.cover_opts(im.IM_RANDGREEDI, P, a, 0.077, 11, False)
    specs = [("a", im.IM_LT, 10, 3000, 5, rg(16, (1, 4))),
             ("b", im.IM_IC, 12, 2500, 6, None),
             ("c", im.IM_LT, 30, 20000, 7, rg(0, (1, 4))),
             ("c", im.IM_LT, 20, 18000, 8, rg(0, (1, 2))),
             ("a", im.IM_LT, 8, 1000, 9, None),
             ("b", im.IM_IC, 5, 4000, 10, rg(32, (1, 1))),
             ("c", im.IM_LT, 25, 20000, 11, im.cover_opts(im.IM_RANDGREEDI, 0, (1, 4), 0.077, 11,
                                                         False, im.IM_AGG_GREEDY))]
    batch = im.im_batch_create()
    try:
        out = im.im_solve_batch(batch, [(G[n].handle, m, k, th, sd, o)
                                        for n, m, k, th, sd, o in specs], 30,
                                with_partitions=True)
    finally:
        im.im_batch_destroy(batch)
    for (name, m, k, th, sd, o), (seeds, gains, cov, entries, parts) in zip(specs, out):
        g = graphs[name]
        mo = O.IC if m == im.IM_IC else O.LT
        pool = O.sample(mo, g, sd, 0, th)
        inv = O.invert(g.n, pool)
        assert entries == pool.members.size
        if o is None:
            r = O.greedy(g.n, pool, inv, k)
            assert parts == 0
        else:
            P = o.partitions or parts
            assert parts == P and P >= 1
            r = O.randgreedi(g.n, pool, inv, k, P, 11, O.trunc_count(k, o.alpha_num, o.alpha_den),
                             0.077, naive=o.aggregator == im.IM_AGG_GREEDY)
        assert seeds.tolist() == r.seeds.tolist(), name
        assert gains.tolist() == r.gains.tolist(), name
        assert cov == r.coverage, name
        if o is not None:                       # the same query alone
            Gp, Pp = gpu_pool(im, g, m, sd, [(0, th)], cap_entries=th * 512)
            alone = Pp.cover(k, im.cover_opts(im.IM_RANDGREEDI, P, (o.alpha_num, o.alpha_den),
                                              0.077, 11, False, o.aggregator))
            assert alone.seeds.tolist() == seeds.tolist() and alone.coverage == cov
            Pp.close()
    for gh in G.values():
        gh.close()


@pytest.mark.parametrize("heavy", [0, 60000])
def test_server_results_equal_alone(im, heavy):
    """Continuous batching: requests submitted back to back land in shared
    batches, and every result equals the oracle's (= the query alone); with a
    heavy lane (the larger requests on worker 0 only, the rest past them)
    as well."""
    import time
    graphs = [inputs.rmat_graph(1 << 12, 1 << 16, 5, "ic0.1"),
              inputs.rmat_graph(1 << 13, 1 << 17, 6, "lt")]
    G = [im.Graph(g) for g in graphs]
    srv = im.im_server_create(workers=3 if heavy else 2, max_batch=16, mem_budget=8 << 30,
                              heavy_members=heavy)
    rng = np.random.default_rng(3)
    reqs = []
    try:
        for r in range(40):
            gi = r % 2
            k = int(rng.integers(1, 30))
            th = int(rng.integers(100, 4000))
            sd = int(rng.integers(0, 2**60))
            t = im.im_server_submit(srv, G[gi].handle, im.IM_IC if gi == 0 else im.IM_LT, k, th, sd)
            reqs.append((t, gi, k, th, sd))
            if r % 7 == 0:
                time.sleep(0.002)
        for t, gi, k, th, sd in reqs:
            seeds, cov, lat = im.im_server_wait(srv, t, 30)
            g = graphs[gi]
            pool = O.sample(O.IC if gi == 0 else O.LT, g, sd, 0, th)
            rc = O.greedy(g.n, pool, O.invert(g.n, pool), k)
            assert seeds.tolist() == rc.seeds.tolist() and cov == rc.coverage
            assert lat > 0
        batches, queries, queued = im.im_server_stats(srv)
        assert queries == 40 and queued == 0 and batches < 40
        with pytest.raises(im.ImError):
            im.im_server_poll(srv, 10**9, 4)      # unknown (or already collected) ticket
    finally:
        im.im_server_destroy(srv)


@pytest.mark.parametrize("replicas", [0, 1, 2, 4, 8])
def test_index_replicas_identical(im, replicas):
    """Every covering-subset build (a tuning knob: radix sort, or counting
    with 1-8 counter replicas) gives the same covering subsets (as sorted
    lists; the radix sort's come out ascending, equal to the oracle's as
    stored) and the same greedy result."""
    old = im.im_tune_get(im.IM_TUNE_INDEX_REPLICAS)
    im.im_tune_set(im.IM_TUNE_INDEX_REPLICAS, replicas)
    try:
        g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
        G, P = gpu_pool(im, g, im.IM_LT, 42, [(0, 40000)])
        ref = O.sample(O.LT, g, 42, 0, 40000)
        assert_index_equal(P, g, ref)
        if replicas == 0:
            vtx_off, set_ids = P.index()
            rv, rs = O.invert(g.n, ref)
            assert np.array_equal(vtx_off, rv) and np.array_equal(set_ids, rs)
        c = P.cover(30)
        rc = O.greedy(g.n, ref, O.invert(g.n, ref), 30)
        assert c.seeds.tolist() == rc.seeds.tolist() and c.coverage == rc.coverage
    finally:
        im.im_tune_set(im.IM_TUNE_INDEX_REPLICAS, old)


@pytest.mark.parametrize("evals", [1, 2, 4, 8])
def test_randgreedi_eval_width_identical(im, evals):
    """Candidates re-evaluated per round in the local greedy (a tuning knob):
    every local solution and bucket stays the oracle's."""
    old = im.im_tune_get(im.IM_TUNE_RG_EVALS)
    im.im_tune_set(im.IM_TUNE_RG_EVALS, evals)
    try:
        g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
        _rg_compare(im, g, im.IM_LT, 30000, 60, 148, (1, 4), 0.077, False)
        _rg_compare(im, g, im.IM_LT, 30000, 20, 7, (1, 1), 0.077, True)
    finally:
        im.im_tune_set(im.IM_TUNE_RG_EVALS, old)


# --- forward simulation (spread of a seed set) -----------------------------------

@pytest.mark.parametrize("model,wmode", [(0, "random"), (0, "0.3"), (0, "one"), (0, "zero"),
                                         (1, "lt"), (1, "lt_random")])
def test_spread_matches_oracle(im, model, wmode):
    """Per-run activated counts and root hits, bit-exact against the oracle's
    forward BFS (duplicated seeds, ragged run counts)."""
    g = inputs.random_graph(60, 400, 13, wmode)
    G = im.Graph(g)
    seeds = np.array([3, 7, 7, 41], np.int32)
    for first, runs in ((0, 1), (5, 33), (1000, 777)):
        act = np.zeros(runs, np.int64)
        hit = np.zeros(runs, np.uint8)
        tot = im.im_spread(G.handle, model, seeds, 21, first, runs, act, hit)
        ra, rh = O.spread(model, g, 21, first, runs, seeds)
        assert np.array_equal(act, ra) and np.array_equal(hit, rh)
        assert tot == int(ra.sum())


def test_spread_rmat_and_ris_identity(im):
    """R-MAT graphs, IC and LT: the oracle's runs bit-exact, and on the device
    the root hits of runs 0..theta-1 add up to the coverage the greedy reports
    for its seeds on the pool of samples 0..theta-1 (two kernels, one world)."""
    import torch
    for model, w, theta in ((im.IM_IC, "ic0.1", 20000), (im.IM_LT, "lt", 50000)):
        g = inputs.rmat_graph(1 << 14, 1 << 18, 42, w)
        G = im.Graph(g)
        P = im.Pool(G, theta, theta * 2048)
        P.sample(model, 42, 0, theta)
        c = P.cover(25)
        hit = torch.zeros(theta, dtype=torch.uint8, device="cuda")
        im.im_spread(G.handle, model, c.seeds, 42, 0, theta, None, hit)
        assert int(hit.sum().item()) == c.coverage
        act = np.zeros(300, np.int64)
        rh = np.zeros(300, np.uint8)
        im.im_spread(G.handle, model, c.seeds, 42, 777, 300, act, rh)
        ra, rrh = O.spread(O.IC if model == im.IM_IC else O.LT, g, 42, 777, 300, c.seeds)
        assert np.array_equal(act, ra) and np.array_equal(rh, rrh)


def test_spread_rejects_bad_seed(im):
    g = inputs.random_graph(30, 100, 2, "0.3")
    G = im.Graph(g)
    with pytest.raises(im.ImError) as e:
        im.im_spread(G.handle, im.IM_IC, np.array([1, 30], np.int32), 1, 0, 10)
    assert e.value.status == im.IM_ERR_INVALID_ARG
    assert im.im_spread(G.handle, im.IM_IC, np.zeros(0, np.int32), 1, 0, 5) == 0


def test_autotune_picks_allowed_values_and_keeps_results(im):
    """im_autotune times the result-invariant knobs on a probe and leaves the
    fastest values set; the pool and both covers still equal the oracle's."""
    knobs = (im.IM_TUNE_LT_GROUP, im.IM_TUNE_RG_CLUSTER, im.IM_TUNE_INDEX_REPLICAS,
             im.IM_TUNE_RG_EVALS, im.IM_TUNE_LT_CACHE, im.IM_TUNE_GREEDY_HOT)
    saved = [im.im_tune_get(kn) for kn in knobs]
    try:
        g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
        G = im.Graph(g)
        opts = im.cover_opts(im.IM_RANDGREEDI, 148, (1, 4), 0.077, 42, False)
        r = im.im_autotune(G.handle, im.IM_LT, 42, 20000, 50, opts)
        assert r["lt_group"] in (1, 8, 16, 32) and r["index_replicas"] in (0, 1, 2, 4, 8)
        assert r["rg_evals"] in (1, 2, 4, 8) and r["rg_cluster"] in (0, 1, 2, 4, 8, -1)
        assert im.im_tune_get(im.IM_TUNE_LT_GROUP) == r["lt_group"]
        assert im.im_tune_get(im.IM_TUNE_RG_CLUSTER) == r["rg_cluster"]
        assert all(x >= 0 for x in r["ms"][0][:4]) and all(x >= 0 for x in r["ms"][3][:6])
        assert r["greedy_hot"] in (0, 7, 8, 10) and all(x >= 0 for x in r["ms"][5][:4])
        assert im.im_tune_get(im.IM_TUNE_GREEDY_HOT) == r["greedy_hot"]
        assert r["lt_cache"] in (-1, 0, 1, 2)
        if r["lt_group"] == 1:
            assert r["lt_cache"] in (0, 1, 2) and all(x >= 0 for x in r["ms"][4][:3])
        _rg_compare(im, g, im.IM_LT, 30000, 50, 148, (1, 4), 0.077, False)
        c = gpu_pool(im, g, im.IM_LT, 42, [(0, 20000)])[1].cover(50)
        ref = O.sample(O.LT, g, 42, 0, 20000)
        rc = O.greedy(g.n, ref, O.invert(g.n, ref), 50)
        assert c.seeds.tolist() == rc.seeds.tolist() and c.coverage == rc.coverage
        G2, P2 = gpu_pool(im, g, im.IM_LT, 7, [(0, 20000)])
        assert_pool_equal(im, P2, O.sample(O.LT, g, 7, 0, 20000))
        r_ic = im.im_autotune(G.handle, im.IM_IC, 3, 5000, 10)
        assert r_ic["lt_group"] == -1 and r_ic["rg_evals"] == -1 and r_ic["lt_cache"] == -1
    finally:
        for kn, v in zip(knobs, saved):
            im.im_tune_set(kn, v)


def test_device_heap_reuse_then_trim(im):
    """Pools created after others were destroyed reuse their cached device
    pages and still give the oracle's sets and the same cover;
    im_trim_memory then hands the cache back to the driver."""
    torch = pytest.importorskip("torch")
    g = inputs.rmat_graph(1 << 12, 1 << 16, 5, "lt")
    ref = oracle_pool(g, 1, 9, [(0, 3000)])
    first = None
    for cap in (1 << 22, 1 << 20, 1 << 23):
        G, P = gpu_pool(im, g, 1, 9, [(0, 3000)], cap_entries=cap)
        assert_pool_equal(im, P, ref)
        c = P.cover(10)
        got = (c.seeds.tolist(), c.gains.tolist(), c.coverage)
        first = first or got
        assert got == first
        P.close()
        G.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    im.im_trim_memory()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0 + (16 << 20)      # the last pool alone cached 2 x 32 MB
    im.im_trim_memory()                      # nothing left to hand back: still ok


def _hub_graph(seed):
    """Hubs 0..7 with in-degrees on both sides of the index build's three
    kernels (one thread up to 32 in-edges, one warp up to 1024, one block of
    2048-edge passes beyond); every other vertex has in-edges from two hubs,
    so LT walks keep passing through the hubs' search trees.  Random LT
    weights with per-vertex sums below 2^32."""
    rng = np.random.default_rng(seed)
    n = 6000
    hub_deg = [33, 1024, 1025, 2047, 2048, 2049, 4097, 5900]
    src, dst = [], []
    for h, d in enumerate(hub_deg):
        s = rng.choice(np.arange(8, n), size=d, replace=False)
        src += s.tolist()
        dst += [h] * d
    for v in range(8, n):
        s = rng.choice(8, size=2, replace=False)
        src += s.tolist()
        dst += [v, v]
    in_off, in_src = inputs.in_csr(n, np.array(src), np.array(dst))
    w = np.zeros(in_src.size, np.uint32)
    for v in range(n):
        b, e = int(in_off[v]), int(in_off[v + 1])
        parts = rng.dirichlet(np.ones(e - b + 1))[: e - b]
        w[b:e] = np.floor(parts * inputs.U32_MAX).astype(np.uint32)
    return inputs.Graph(n, in_off, in_src, w)


def test_lt_index_hub_degrees_match_oracle(im):
    g = _hub_graph(17)
    ids = [(0, 12000), (12000, 8000)]
    G, P = gpu_pool(im, g, im.IM_LT, 23, ids, cap_entries=1 << 24)
    assert im.im_graph_info(G.handle)[2] == 1
    assert_pool_equal(im, P, oracle_pool(g, 1, 23, ids))


@pytest.mark.parametrize("hub", [1, 5])       # in-degree 1024 (warp), 2049 (block)
def test_lt_index_flags_weights_above_one(im, hub):
    g = _hub_graph(17)
    w = g.w.copy()
    b, e = int(g.in_off[hub]), int(g.in_off[hub + 1])
    w[b:e] = np.uint32(1 << 23)               # sum (e - b) 2^23 > 2^32
    G = im.Graph(inputs.Graph(g.n, g.in_off, g.in_src, w))
    assert im.im_graph_info(G.handle)[2] == 0


@pytest.mark.parametrize("seed", [3, 4])
def test_lt_equal_weight_vertices_mixed_with_unequal(im, seed):
    """Vertices whose in-edges all weigh the same u take the pick from
    floor(x / u) instead of the cut-point table; here every other vertex has
    equal weights whose sum d u stays below 2^32 by a random margin (so some
    draws pick nothing), the rest random weights, over the hub graph's
    in-degrees (index built by thread, warp and block)."""
    g = _hub_graph(seed)
    rng = np.random.default_rng(seed + 100)
    w = g.w.copy()
    for v in range(0, g.n, 2):
        b, e = int(g.in_off[v]), int(g.in_off[v + 1])
        if e > b:
            total = rng.uniform(0.3, 1.0) * inputs.U32_MAX
            w[b:e] = np.uint32(max(1, int(total // (e - b))))
    g = inputs.Graph(g.n, g.in_off, g.in_src, w)
    ids = [(0, 9000), (9000, 3001)]
    G, P = gpu_pool(im, g, im.IM_LT, 77, ids, cap_entries=1 << 24)
    assert im.im_graph_info(G.handle)[2] == 1
    ref = oracle_pool(g, 1, 77, ids)
    assert_pool_equal(im, P, ref)
    assert_index_equal(P, g, ref)


def test_ic_giant_sets_through_hubs(im):
    """Giant sets (second pass, one block per set) that pass through hubs of
    4,096 to 20,011 in-edges with unaligned first edges, reached from every
    root (every vertex has in-edges from three hubs)."""
    rng = np.random.default_rng(12)
    n = 30000
    hub_deg = [4096, 4097, 5001, 9000, 20011, 4099 * 4 + 3]
    src, dst = [], []
    for h, d in enumerate(hub_deg):
        s = rng.choice(np.arange(len(hub_deg), n), size=d, replace=False)
        src += s.tolist()
        dst += [h] * d
    for v in range(len(hub_deg), n):
        hs = rng.choice(len(hub_deg), size=3, replace=False)
        rs = rng.integers(len(hub_deg), n, size=2)
        for u in set(hs.tolist() + rs.tolist()) - {v}:
            src.append(u)
            dst.append(v)
    in_off, in_src = inputs.in_csr(n, np.array(src), np.array(dst))
    w = np.full(in_src.size, np.uint32(int(0.9 * inputs.U32_MAX)))
    g = inputs.Graph(n, in_off, in_src, w)
    G, P = gpu_pool(im, g, im.IM_IC, 31, [(0, 150), (150, 61)], cap_entries=211 * n)
    ref = oracle_pool(g, O.IC, 31, [(0, 150), (150, 61)])
    assert np.diff(ref.set_off).max() > 16384
    assert_pool_equal(im, P, ref)
