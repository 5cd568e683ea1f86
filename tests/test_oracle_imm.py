"""Structure of the oracle's IMM driver (Alg. 1).  The formulas themselves are
not in the paper (it defers them to Tang et al. 2015): parity unpinned; these
tests check the structure Alg. 1 fixes."""
import itertools
import math

import numpy as np
import pytest

from oracle import brute, imm
from paper_2408_10982_gb300 import inputs


def test_constants_shape(orc):
    c = imm.constants(4847571, 200, 0.13, 1.0)
    assert c["rounds"] == int(math.floor(math.log2(4847571))) - 1
    assert c["eps2"] == np.sqrt(2) * 0.13
    assert c["lambda_star"] > c["lambda_prime"] > 0
    # smaller eps, more samples; larger k, more samples
    assert imm.constants(10000, 10, 0.1, 1)["lambda_star"] > imm.constants(10000, 10, 0.2, 1)["lambda_star"]
    assert imm.constants(10000, 20, 0.1, 1)["lambda_star"] > imm.constants(10000, 10, 0.1, 1)["lambda_star"]


def test_imm_rounds_double_and_stop(orc):
    g = inputs.rmat_graph(4096, 65536, 7, "trivalency")
    r = imm.imm(g, orc.IC, 10, 0.5, 1.0, 42)
    c = imm.constants(g.n, 10, 0.5, 1.0)
    # theta_i = ceil(lambda' / (n / 2^i)): each round (about) doubles the pool
    for i, th in enumerate(r.theta_rounds, start=1):
        assert th == math.ceil(c["lambda_prime"] / (g.n / 2 ** i))
    for a, b in zip(r.theta_rounds, r.theta_rounds[1:]):
        assert 2 * a - 1 <= b <= 2 * a + 1
    assert r.lb >= 1.0
    assert r.theta == math.ceil(c["lambda_star"] / r.lb)
    assert len(r.seeds) <= 10 and r.coverage > 0


@pytest.mark.parametrize("n,m,p,gseed", [(12, 11, "0.9", 2), (12, 11, "0.9", 3),
                                         (10, 11, "0.8", 2), (10, 12, "0.7", 1)])
def test_imm_seeds_meet_the_papers_guarantee(orc, n, m, p, gseed):
    """The paper's restated IMM theorem (Sec. 2.2): the seeds are within
    (1 - 1/e - eps) of the optimal expected influence with probability at least
    1 - 1/n^l.  sigma is exact (every IC live-edge world of an 11- or 12-edge
    graph), OPT by enumerating every k-subset; on these graphs 15 to 28 of the
    45 or 66 seed pairs fall below the bound."""
    g = inputs.random_graph(n, m, gseed, p)
    k, eps = 2, 0.1
    r = imm.imm(g, orc.IC, k, eps, 1.0, 42)
    opt = max(brute.ic_spread_exact(g, list(S)) for S in itertools.combinations(range(g.n), k))
    got = brute.ic_spread_exact(g, [int(v) for v in r.seeds])
    assert float(got) >= (1 - 1 / math.e - eps) * float(opt)
