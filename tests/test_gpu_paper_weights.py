"""The paper's own weight model (Sec. 4.1: edge probabilities drawn U[0, 0.1])
through the GPU path against the oracle: IC sampling, the LT variant (the same
draws, each vertex's in-weights scaled to sum to at most 1), covering subsets,
the greedy and RandGreedi (streaming and non-streaming global step).  Integer
results: the bar is equality."""
import numpy as np
import pytest

import oracle as O
from paper_2408_10982_gb300 import inputs

from test_gpu_parity import _rg_compare, assert_index_equal, assert_pool_equal, gpu_pool

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


@pytest.mark.parametrize("model,wts,theta", [("ic", "u0.1", 1024), ("lt", "lt-u0.1", 50000)])
def test_paper_weights_pool_index_and_greedy(im, model, wts, theta):
    g = inputs.rmat_graph(1 << 16, 1 << 20, 42, wts)
    m = im.IM_IC if model == "ic" else im.IM_LT
    mo = O.IC if model == "ic" else O.LT
    G, P = gpu_pool(im, g, m, 7, [(0, theta)], cap_entries=theta * 65536)
    ref = O.sample(mo, g, 7, 0, theta)
    assert_pool_equal(im, P, ref)
    assert_index_equal(P, g, ref)
    inv = O.invert(g.n, ref)
    for k in (1, 50):
        c = P.cover(k)
        rc = O.greedy(g.n, ref, inv, k)
        assert c.seeds.tolist() == rc.seeds.tolist() and c.gains.tolist() == rc.gains.tolist()
        assert c.coverage == rc.coverage
    P.close()
    G.close()


@pytest.mark.parametrize("naive", [False, True])
@pytest.mark.parametrize("model,wts,theta", [("ic", "u0.1", 1024), ("lt", "lt-u0.1", 30000)])
def test_paper_weights_randgreedi(im, model, wts, theta, naive):
    g = inputs.rmat_graph(1 << 16, 1 << 20, 42, wts)
    m = im.IM_IC if model == "ic" else im.IM_LT
    _rg_compare(im, g, m, theta, 50, 148, (1, 4), 0.077, False, seed=5, naive=naive)


def test_paper_weights_scale20_ic_sampled_ids(im):
    """R-MAT scale 20 with U[0, 0.1] IC probabilities (15% of sets hold a
    ~10^5-vertex giant component): 32 sets at ids spread over [0, 2^22)
    against the oracle one by one."""
    g = inputs.rmat_graph(1 << 20, 1 << 24, 42, "u0.1")
    G = im.Graph(g)
    rng = np.random.default_rng(3)
    firsts = sorted(int(x) for x in rng.choice(1 << 21, size=16, replace=False) * 2)
    pool = im.Pool(G, 32, 32 * g.n)
    for f in firsts:
        pool.sample(im.IM_IC, 42, f, 2)
    set_off, members = pool.export()
    ex = 0
    for i, f in enumerate(firsts):
        ref = O.sample(O.IC, g, 42, f, 2)
        ex += ref.examined
        for t in range(2):
            s = 2 * i + t
            assert np.array_equal(members[set_off[s]:set_off[s + 1]], ref.set(t)), (f, t)
    assert pool.info()[2] == ex
    pool.close()
    G.close()
