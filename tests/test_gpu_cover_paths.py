"""The alternative max-k-cover paths on the GPU against the oracle: the lazy
greedy of Alg. 2 (IM_GREEDY_LAZY, and IM_GREEDY_PLAIN run by the lazy kernel)
and RandGreedi with Alg. 4's non-streaming global step (IM_AGG_GREEDY).
Seeds, gains and coverage are integers: the bar is equality."""
import numpy as np
import pytest

import oracle as O
from paper_2408_10982_gb300 import inputs

from test_gpu_parity import _rg_compare, gpu_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def im():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_10982_gb300 import build, im as imm
    build.build_library()
    O.build()
    yield imm
    imm.im_tune_set(imm.IM_TUNE_GREEDY_EVALS, 0)


def _lazy_vs_oracle(im, g, model, seed, theta, k, widths=(1, 2, 4, 8, 16, 32)):
    G, P = gpu_pool(im, g, model, seed, [(0, theta)])
    ref = O.sample(model, g, seed, 0, theta)
    inv = O.invert(g.n, ref)
    rc = O.greedy(g.n, ref, inv, k)
    rl = O.lazy_greedy(g.n, ref, inv, k)
    assert rl.seeds.tolist() == rc.seeds.tolist() and rl.coverage == rc.coverage
    stats = []
    for W in widths:
        im.im_tune_set(im.IM_TUNE_GREEDY_EVALS, W)
        for algo in (im.IM_GREEDY_LAZY, im.IM_GREEDY_PLAIN):
            c = P.cover(k, im.cover_opts(algo))
            assert c.seeds.tolist() == rc.seeds.tolist(), (W, algo)
            assert c.gains.tolist() == rc.gains.tolist(), (W, algo)
            assert c.coverage == rc.coverage, (W, algo)
            stats.append(im.im_greedy_stats(P.handle))
    im.im_tune_set(im.IM_TUNE_GREEDY_EVALS, 0)
    c = P.cover(k)                                  # the counts-decrement kernel
    assert c.seeds.tolist() == rc.seeds.tolist() and c.coverage == rc.coverage
    P.close()
    G.close()
    return stats


def test_lazy_small_ic_full(im):
    _lazy_vs_oracle(im, inputs.graph_small_ic(), im.IM_IC, 42, 16384, 16)


@pytest.mark.parametrize("k", [1, 7, 100])
def test_lazy_rmat_lt(im, k):
    g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
    _lazy_vs_oracle(im, g, im.IM_LT, 7, 20000, k)


@pytest.mark.parametrize("theta", [1, 3, 40])
def test_lazy_tie_heavy(im, theta):
    """Few sets: almost every gain ties, the smallest id must win every tie."""
    g = inputs.rmat_graph(1 << 12, 1 << 16, 3, "lt")
    _lazy_vs_oracle(im, g, im.IM_LT, 9, theta, 50, widths=(1, 4, 32))


def test_lazy_rebuilds_its_bound_list(im):
    """More than 8,192 vertices with a positive bound and picks down to gain 1:
    the top-8,192 list is built with ties split by id, runs dry and is rebuilt
    from the bounds array; the seeds still equal the oracle's."""
    g = inputs.rmat_graph(1 << 16, 1 << 20, 42, "lt")
    stats = _lazy_vs_oracle(im, g, im.IM_LT, 42, 2000, 400, widths=(4, 32))
    assert all(s["builds"] >= 2 for s in stats), stats


def test_lazy_zero_gain_stop_and_empty_pool(im):
    g = inputs.random_graph(30, 60, 2, "zero")      # every set is a singleton
    _lazy_vs_oracle(im, g, im.IM_IC, 3, 10, 25, widths=(1, 8))
    G = im.Graph(inputs.random_graph(30, 60, 2, "0.5"))
    P = im.Pool(G, 10, 100)
    for algo in (im.IM_GREEDY_LAZY,):
        c = P.cover(5, im.cover_opts(algo))
        assert len(c.seeds) == 0 and c.coverage == 0
    P.close()
    G.close()


def test_lazy_full_size_rmat20(im):
    """The benchmark workload (R-MAT scale 20, LT, theta = 4,194,304, k = 100)
    on the first 1,048,576 sets: the lazy greedy equals the oracle's greedy."""
    from oracle import parallel
    g = inputs.graph_lt_scale20(42)
    theta, k = 1 << 20, 100
    G, P = gpu_pool(im, g, im.IM_LT, 42, [(0, theta)], cap_entries=theta * 64)
    ref = parallel.sample(O.LT, g, 42, 0, theta)
    rc = O.greedy(g.n, ref, O.invert(g.n, ref), k)
    for W in (4, 32):
        im.im_tune_set(im.IM_TUNE_GREEDY_EVALS, W)
        c = P.cover(k, im.cover_opts(im.IM_GREEDY_LAZY))
        assert c.seeds.tolist() == rc.seeds.tolist() and c.gains.tolist() == rc.gains.tolist()
        assert c.coverage == rc.coverage
    im.im_tune_set(im.IM_TUNE_GREEDY_EVALS, 0)
    P.close()
    G.close()


@pytest.mark.parametrize("Pn,alpha,k", [(148, (1, 4), 100), (7, (1, 1), 20), (1, (1, 2), 20),
                                        (32, (1, 8), 50)])
def test_randgreedi_naive_aggregator_lt(im, Pn, alpha, k):
    g = inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt")
    _rg_compare(im, g, im.IM_LT, 30000, k, Pn, alpha, 0.077, False, naive=True)


def test_randgreedi_naive_aggregator_ic_small(im):
    _rg_compare(im, inputs.graph_small_ic(), im.IM_IC, 16384, 16, 16, (1, 2), 0.1, False,
                naive=True)


def test_randgreedi_naive_rejects_bad_aggregator(im):
    g = inputs.graph_small_ic()
    G, P = gpu_pool(im, g, im.IM_IC, 42, [(0, 100)])
    opts = im.cover_opts(im.IM_RANDGREEDI, 4, (1, 1), 0.1, 1, False, 7)
    with pytest.raises(im.ImError) as e:
        P.cover(4, opts)
    assert e.value.status == im.IM_ERR_INVALID_ARG


@pytest.mark.parametrize("shift", [0, 4, 8, 16])
def test_greedy_hot_vertex_threshold(im, shift):
    """The standard greedy with exact gains kept only for vertices with
    |S(v)| >= max |S(v)| >> shift: the seeds equal the oracle's, including
    instances whose best gain falls below that bound (tau = l/16 on k = 100
    picks), where the stale gains are made exact midway."""
    im.im_tune_set(im.IM_TUNE_GREEDY_HOT, shift)
    try:
        cases = [(inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt"), im.IM_LT, 20000, 100),
                 (inputs.graph_small_ic(), im.IM_IC, 16384, 16),
                 (inputs.rmat_graph(1 << 12, 1 << 16, 3, "lt"), im.IM_LT, 40, 50)]
        for g, model, theta, k in cases:
            G, P = gpu_pool(im, g, model, 7, [(0, theta)], cap_entries=theta * 1024)
            ref = O.sample(O.IC if model == im.IM_IC else O.LT, g, 7, 0, theta)
            rc = O.greedy(g.n, ref, O.invert(g.n, ref), k)
            c = P.cover(k)
            assert c.seeds.tolist() == rc.seeds.tolist() and c.gains.tolist() == rc.gains.tolist()
            assert c.coverage == rc.coverage
            P.close()
            G.close()
    finally:
        im.im_tune_set(im.IM_TUNE_GREEDY_HOT, 8)
