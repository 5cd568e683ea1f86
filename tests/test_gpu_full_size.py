"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times (default knobs: one LT walk per thread, RandGreedi in two
launches with the bucket-mask stage).

R-MAT scale 20, LT 1/in-degree, theta = 4,194,304, k = 100: every RRR set, the
plain greedy and RandGreedi (148 parts, alpha = 1/4, delta = 0.077; every
local solution and every bucket) against the oracle, element by element.  The
oracle samples its sets over spawned worker processes (`oracle.parallel`;
sample ids key every draw, so the split does not change them).

LiveJournal-shaped R-MAT (4,847,571 vertices, 69,000,000 edges, IC
trivalency): sets at sampled ids spread over [0, 2^24), each computed by the
oracle one by one.
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


def test_rmat20_lt_full_pool_greedy_and_randgreedi(im):
    from oracle import parallel
    theta, k, P, alpha, delta, seed = 4_194_304, 100, 148, (1, 4), 0.077, 42
    g = inputs.graph_lt_scale20(seed)
    G = im.Graph(g)
    pool = im.Pool(G, theta, theta * 64)
    pool.sample(im.IM_LT, seed, 0, theta)
    set_off, members = pool.export()
    ref = parallel.sample(O.LT, g, seed, 0, theta)
    assert np.array_equal(set_off, ref.set_off)
    assert np.array_equal(members, ref.members)
    assert pool.info()[2] == ref.examined
    inv = O.invert(g.n, ref)

    c = pool.cover(k)
    rc = O.greedy(g.n, ref, inv, k)
    assert c.seeds.tolist() == rc.seeds.tolist()
    assert c.gains.tolist() == rc.gains.tolist()
    assert c.coverage == rc.coverage

    trunc = O.trunc_count(k, *alpha)
    r = O.randgreedi(g.n, ref, inv, k, P, seed, trunc, delta)
    opts = im.cover_opts(im.IM_RANDGREEDI, P, alpha, delta, seed, fused=False)
    c = pool.cover(k, opts)
    B = O.num_buckets(k, delta)
    d = pool.randgreedi_details(k, P, B)
    assert np.array_equal(d["local_n"], r.local_n)
    assert np.array_equal(d["local_cov"], r.local_cov)
    for p in range(P):
        n_p = r.local_n[p]
        assert d["local_seeds"][p, :n_p].tolist() == r.local_seeds[p, :n_p].tolist(), p
        assert d["local_gains"][p, :n_p].tolist() == r.local_gains[p, :n_p].tolist(), p
    assert np.array_equal(d["thr"], r.thr)
    assert np.array_equal(d["bucket_n"], r.buckets.n)
    assert np.array_equal(d["bucket_cov"], r.buckets.cov)
    for b in range(B):
        nb = r.buckets.n[b]
        assert d["bucket_seeds"][b, :nb].tolist() == r.buckets.seeds[b, :nb].tolist(), b
        assert d["bucket_gains"][b, :nb].tolist() == r.buckets.gains[b, :nb].tolist(), b
    assert d["chosen"] == r.chosen
    assert c.seeds.tolist() == r.seeds.tolist()
    assert c.coverage == r.coverage
    pool.close()
    G.close()


def test_livejournal_shaped_ic_sampled_ids(im):
    """IC trivalency on the LiveJournal-shaped graph: 48 sets at ids spread over
    [0, 2^24) (ranges of 2 ids), appended to one pool, against the oracle."""
    g = inputs.graph_livejournal_like(42)
    G = im.Graph(g)
    rng = np.random.default_rng(7)
    firsts = sorted(int(x) for x in rng.choice(1 << 23, size=24, replace=False) * 2)
    ids = [(f, 2) for f in firsts]
    pool = im.Pool(G, 48, 48 * g.n)
    for f, c in ids:
        pool.sample(im.IM_IC, 42, f, c)
    set_off, members = pool.export()
    ex = 0
    for i, (f, c) in enumerate(ids):
        ref = O.sample(O.IC, g, 42, f, c)
        ex += ref.examined
        for t in range(c):
            s = 2 * i + t
            got = members[set_off[s]:set_off[s + 1]]
            assert np.array_equal(got, ref.set(t)), (f, t)
    assert pool.info()[2] == ex
    pool.close()
    G.close()


def _solve_alone(im, G, model, k, theta, seed, cap_per_set=64):
    """The one-query path: im_sample_rrr into a fresh pool, then plain greedy."""
    while True:
        pool = im.Pool(G, max(theta, 1), max(theta, 1) * cap_per_set)
        try:
            pool.sample(model, seed, 0, theta)
        except im.ImError as e:
            pool.close()
            if e.status != im.IM_ERR_CAPACITY:
                raise
            cap_per_set *= 4
            continue
        c = pool.cover(k)
        entries = pool.info()[1]
        pool.close()
        return c.seeds, c.gains, c.coverage, entries


def test_batched_mix_256_queries(im):
    """The batched workload (256 queries over R-MAT scales 12..18, IC weighted
    cascade or LT, k in [5, 100], theta in [2^14, 2^20]) in one im_solve_batch
    call: every query equals the one-query path; the six smallest queries and
    the smallest of every (scale, model) pair equal the oracle."""
    specs = inputs.batched_queries(256, 42)
    graphs = {f"rmat{s}": inputs.batched_graph(s, 42) for s in inputs.BATCH_SCALES}
    G = {name: im.Graph(g) for name, g in graphs.items()}
    batch = im.im_batch_create()
    try:
        out = im.im_solve_batch(batch, [(G[q.graph].handle, q.model, q.k, q.theta, q.seed)
                                        for q in specs], 100)
    finally:
        im.im_batch_destroy(batch)
    for q, (seeds, gains, cov, entries) in zip(specs, out):
        s1, g1, c1, e1 = _solve_alone(im, G[q.graph], q.model, q.k, q.theta, q.seed)
        assert seeds.tolist() == s1.tolist(), q
        assert gains.tolist() == g1.tolist(), q
        assert cov == c1 and entries == e1, q
    order = sorted(range(len(specs)), key=lambda i: (specs[i].theta << 8) + int(specs[i].graph[4:]))
    picked, seen = list(order[:6]), set()
    for i in order:                         # the smallest query of every (scale, model)
        key = (specs[i].graph, specs[i].model)
        if key not in seen:
            seen.add(key)
            if i not in picked:
                picked.append(i)
    for i in picked:
        q = specs[i]
        g = graphs[q.graph]
        pool = O.sample(q.model, g, q.seed, 0, q.theta)
        rc = O.greedy(g.n, pool, O.invert(g.n, pool), q.k)
        seeds, gains, cov, entries = out[i]
        assert seeds.tolist() == rc.seeds.tolist(), q
        assert gains.tolist() == rc.gains.tolist(), q
        assert cov == rc.coverage and entries == pool.members.size, q


@pytest.mark.parametrize("workers,heavy", [(2, 0), (3, 1 << 22)])
def test_served_trace_results_equal_alone(im, workers, heavy):
    """Continuous batching on the served trace (Poisson arrivals, mean 200/s,
    queries drawn like the batched mix): requests are submitted at their
    arrival times while earlier ones run, and every served result equals the
    one-query path; with a heavy lane as well (the largest queries alone on
    worker 0, the rest batched by the others)."""
    import time
    specs = inputs.served_trace(256, 42, orkut_frac=0.0)
    graphs = {f"rmat{s}": inputs.batched_graph(s, 42) for s in inputs.BATCH_SCALES}
    G = {name: im.Graph(g) for name, g in graphs.items()}
    srv = im.im_server_create(workers=workers, max_batch=64, mem_budget=96 << 30,
                              heavy_members=heavy)
    tickets = []
    try:
        t0 = time.perf_counter()
        for q in specs:
            delay = q.arrival_s - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(im.im_server_submit(srv, G[q.graph].handle, q.model, q.k, q.theta,
                                               q.seed))
        results = [im.im_server_wait(srv, t, 100, 600) for t in tickets]
        batches, queries, queued = im.im_server_stats(srv)
    finally:
        im.im_server_destroy(srv)
    assert queries == len(specs) and queued == 0
    assert 1 < batches < len(specs)             # requests were batched, not run one by one
    for q, (seeds, cov, lat) in zip(specs, results):
        s1, _, c1, _ = _solve_alone(im, G[q.graph], q.model, q.k, q.theta, q.seed)
        assert seeds.tolist() == s1.tolist(), q
        assert cov == c1, q
        assert lat > 0


def test_rmat20_lt_spread_of_greedy_seeds(im):
    """The bench workload's plain-greedy seeds (on the first 65,536 sets): the
    root hits of the forward runs over sample ids 0..4095 equal the seeds'
    coverage of those sets in the oracle's pool, and two runs equal the
    oracle's forward BFS (each run activates ~10^5 vertices)."""
    theta, k, seed, runs = 65536, 100, 42, 4096
    g = inputs.graph_lt_scale20(seed)
    G = im.Graph(g)
    pool = im.Pool(G, theta, theta * 64)
    pool.sample(im.IM_LT, seed, 0, theta)
    seeds = pool.cover(k).seeds
    hit = np.zeros(runs, np.uint8)
    im.im_spread(G.handle, im.IM_LT, seeds, seed, 0, runs, None, hit)
    ref = O.sample(O.LT, g, seed, 0, runs)
    S = set(int(x) for x in seeds)
    cov = np.array([1 if S & set(int(v) for v in ref.set(i)) else 0 for i in range(runs)], np.uint8)
    assert np.array_equal(hit, cov)
    act = np.zeros(2, np.int64)
    im.im_spread(G.handle, im.IM_LT, seeds, seed, 1 << 30, 2, act, None)
    ra, _ = O.spread(O.LT, g, seed, 1 << 30, 2, seeds)
    assert np.array_equal(act, ra)
    pool.close()
    G.close()


def _pool_sets(im, handle, n):
    theta, total, _ = im.im_pool_info(handle)
    set_off = np.zeros(theta + 1, np.int64)
    members = np.zeros(max(total, 1), np.int32)
    im.im_pool_export(handle, set_off, members)
    return set_off, members[:total]


def test_imm_at_the_livejournal_size(im):
    """IMM (Alg. 1) as configured for the LiveJournal-shaped graph: eps = 0.13,
    l = 1, k = 200, IC weighted cascade (4,847,571 vertices, 69,000,000 edges).
    Against the oracle: every round's theta_i, each round's CheckGoodness
    decision and LB from the coverage it reached, the final theta = ceil(lambda*
    / LB); sets at the start and the end of the rounds' pool and of the final
    pool (the final pool's ids continue after the rounds'), each computed by
    the oracle; and, on the whole final pool, that the reported coverage is the
    number of sets that contain a seed and that the first seed is a vertex in
    the most sets."""
    import ctypes
    from oracle import imm as OI
    g = inputs.graph_livejournal_like_both(42)["wc"]
    n, k, eps, ell, seed = g.n, 200, 0.13, 1.0, 42
    G = im.Graph(g)
    seeds, cov, theta, info = im.im_solve(G.handle, im.IM_IC, k, eps, ell, seed, keep_pools=True)
    try:
        c = OI.constants(n, k, eps, ell)
        lib = OI._imm_lib()
        assert 1 <= info.rounds <= c["rounds"]
        lb = 1.0
        for i in range(1, info.rounds + 1):
            th = int(lib.orc_imm_round_theta(c["lambda_prime"], n, i))
            assert info.theta_rounds[i - 1] == th
            out = ctypes.c_double(0.0)
            passed = lib.orc_imm_check(n, int(info.cov_rounds[i - 1]), th, i, c["eps2"],
                                       ctypes.byref(out))
            assert passed == (1 if i == info.rounds and info.lb != 1.0 else 0), i
            if passed:
                lb = out.value
        assert info.lb == lb
        assert theta == info.theta == int(lib.orc_imm_final_theta(c["lambda_star"], lb))
        last = int(info.theta_rounds[info.rounds - 1])

        # the rounds' pool holds ids 0 .. last-1, the final pool the next theta ids
        r_off, r_mem = _pool_sets(im, info.round_pool, n)
        f_off, f_mem = _pool_sets(im, info.final_pool, n)
        assert r_off.size - 1 == last and f_off.size - 1 == theta
        assert r_mem.size == info.round_entries and f_mem.size == info.final_entries
        for off, mem, first, ids in ((r_off, r_mem, 0, [(0, 768), (last - 256, 256)]),
                                     (f_off, f_mem, last, [(0, 768), (theta - 256, 256)])):
            for a, cnt in ids:
                ref = O.sample(O.IC, g, seed, first + a, cnt)
                got_off = off[a:a + cnt + 1] - off[a]
                assert np.array_equal(got_off, ref.set_off), (first, a)
                assert np.array_equal(mem[off[a]:off[a + cnt]], ref.members), (first, a)

        # the final answer, on the whole final pool
        assert 1 <= len(seeds) <= k and len(set(seeds.tolist())) == len(seeds)
        is_seed = np.zeros(n, bool)
        is_seed[seeds] = True
        set_of = np.repeat(np.arange(theta), np.diff(f_off))
        hit = np.zeros(theta, bool)
        hit[set_of[is_seed[f_mem]]] = True
        assert cov == int(hit.sum())
        deg = np.bincount(f_mem, minlength=n)
        assert deg[seeds[0]] == deg.max() and seeds[0] == int(np.argmax(deg))
    finally:
        for h in (info.round_pool, info.final_pool):
            if h:
                im.im_pool_destroy(h)
        G.close()
