"""im_opim (OPIM rounds with GreediRIS seed selection, Sec. 3.3.2 / Sec. 4.4)
against the oracle's OPIM driver: every round's theta, the seeds' coverage of
R1 and of R2, the upper bound on the optimum's coverage, and the guarantee --
integers equal, the doubles computed by the same closed forms in the same
order (so equal to the bit)."""
import numpy as np
import pytest

import oracle as O
from oracle import opim as OP
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


def _compare(im, g, model, k, eps, delta, cap, rg):
    opts = None
    rgo = None
    if rg:
        P, alpha = rg
        opts = im.cover_opts(im.IM_RANDGREEDI, P, alpha, 0.1, 9, False)
        rgo = (P, 9, O.trunc_count(k, *alpha), 0.1)
    ref = OP.opim(g, O.IC if model == im.IM_IC else O.LT, k, eps, delta, 42, cap, rgo)
    G = im.Graph(g)
    seeds, info = im.im_opim(G.handle, model, k, eps, delta, 42, cap, opts)
    r = info.rounds
    assert list(info.theta[:r]) == ref.thetas
    assert list(info.cov1[:r]) == ref.cov1
    assert list(info.cov2[:r]) == ref.cov2
    assert list(info.cov1_upper[:r]) == ref.cov1u
    assert list(info.alpha[:r]) == ref.alphas
    assert info.sigma_lower == ref.sigma_l and info.sigma_upper == ref.sigma_u
    assert seeds.tolist() == ref.seeds.tolist()
    G.close()
    return info


@pytest.mark.parametrize("model,wts", [("ic", "trivalency"), ("lt", "lt")])
@pytest.mark.parametrize("rg", [None, (16, (1, 2))])
def test_opim_matches_oracle(im, model, wts, rg):
    g = inputs.rmat_graph(4096, 65536, 7, wts)
    m = im.IM_IC if model == "ic" else im.IM_LT
    info = _compare(im, g, m, 10, 0.3, 1.0 / 4096, 1 << 16, rg)
    assert info.rounds >= 1 and 0 < info.guarantee <= 1


def test_opim_stops_at_the_target(im):
    """A loose eps: the rounds stop as soon as the guarantee reaches 1-1/e-eps."""
    g = inputs.rmat_graph(4096, 65536, 3, "lt")
    info = _compare(im, g, im.IM_LT, 5, 0.5, 0.01, 0, None)
    r = info.rounds
    assert info.alpha[r - 1] >= 1 - np.exp(-1) - 0.5
    assert all(a < 1 - np.exp(-1) - 0.5 for a in info.alpha[: r - 1])


def _sets(im, handle):
    theta, total, _ = im.im_pool_info(handle)
    so = np.zeros(theta + 1, np.int64)
    mem = np.zeros(max(total, 1), np.int32)
    im.im_pool_export(handle, so, mem)
    return so, mem[:total]


def test_opim_at_the_bench_size(im):
    """R-MAT scale 20, LT, k = 1000, eps = 0.01, delta = 1/n, halves capped at
    2^20 sets, GreediRIS-trunc (148 parts, alpha = 1/4, delta_b = 0.0562):
    thetas from the oracle's constants, sets at the start and the end of both
    halves against the oracle, cov2 recomputed from the exported R2 and the
    seeds, and each round's guarantee from the reported counts by the oracle's
    bounds."""
    g = inputs.graph_lt_scale20(42)
    n, k, eps, delta, cap = g.n, 1000, 0.01, 1.0 / g.n, 1 << 20
    opts = im.cover_opts(im.IM_RANDGREEDI, 148, (1, 4), 0.0562, 42, False)
    G = im.Graph(g)
    seeds, info = im.im_opim(G.handle, im.IM_LT, k, eps, delta, 42, cap, opts, keep_pools=True)
    try:
        c = OP.constants(n, k, eps, delta, cap)
        assert info.theta0 == c["theta0"] and info.max_rounds == c["rounds"] and info.a == c["a"]
        r = info.rounds
        assert list(info.theta[:r]) == [c["theta0"] << i for i in range(r)]
        for i in range(r):
            th = int(info.theta[i])
            sl = OP.lower(int(info.cov2[i]), th, n, c["a"])
            su = OP.upper(int(info.cov1_upper[i]), th, n, c["a"])
            assert info.alpha[i] == sl / su
            assert info.cov1_upper[i] >= info.cov1[i]
        th = int(info.theta[r - 1])
        for h, first in ((info.r1_pool, 0), (info.r2_pool, OP.R2_FIRST)):
            so, mem = _sets(im, h)
            assert so.size - 1 == th
            for a, cnt in ((0, 512), (th - 512, 512)):
                ref = O.sample(O.LT, g, 42, first + a, cnt)
                assert np.array_equal(so[a:a + cnt + 1] - so[a], ref.set_off)
                assert np.array_equal(mem[so[a]:so[a + cnt]], ref.members)
        so, mem = _sets(im, info.r2_pool)
        is_seed = np.zeros(n, bool)
        is_seed[seeds] = True
        hit = np.zeros(th, bool)
        hit[np.repeat(np.arange(th), np.diff(so))[is_seed[mem]]] = True
        assert int(hit.sum()) == info.cov2[r - 1]
        assert 1 <= len(seeds) <= k and 0 < info.guarantee <= 1
    finally:
        for h in (info.r1_pool, info.r2_pool):
            if h:
                im.im_pool_destroy(h)
        G.close()
