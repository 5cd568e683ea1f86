"""Pins of the oracle's OPIM driver (oracle/opim.py; the formulas in oracle.c).

The paper runs GreediRIS inside OPIM (Sec. 3.3.2, Sec. 4.4, Table 6) but
prints none of OPIM's formulas (they are Tang et al. 2018's).  They are pinned
here by what they are derived from: each confidence bound is the root of its
martingale tail equation (checked by substitution, not by retyping the closed
form); theta_max spends the final failure budget exactly like IMM's lambda*
with OPT >= k; the budget a splits delta over three events and i_max rounds;
and, on tiny graphs, the reported guarantee is checked against the exact
spread of the selected seeds and the exact optimum."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import brute, opim
from paper_2408_10982_gb300 import inputs


@pytest.mark.parametrize("cov2,theta,n,a", [(0, 100, 1000, 5.0), (37, 1000, 5000, 12.3),
                                           (123456, 1 << 20, 1 << 20, 16.9),
                                           (5, 10, 10, 0.7)])
def test_lower_bound_is_the_root_of_the_upper_tail(orc, cov2, theta, n, a):
    """sigma_l n/theta... rescaled: x = sigma_l theta / n must satisfy
    cov2 = x + a/3 + sqrt(a^2/9 + 2 a x): the coverage exceeds its mean x by
    the Bernstein deviation of budget e^-a exactly."""
    x = opim.lower(cov2, theta, n, a) * theta / n
    r = math.sqrt((cov2 + 2 * a / 9)) - math.sqrt(a / 2)
    if r < 0 or x < 0:            # no positive root: the bound carries no information
        assert x <= 0 or cov2 == 0
        return
    assert math.isclose(x + a / 3 + math.sqrt(a * a / 9 + 2 * a * x), cov2, rel_tol=1e-12,
                        abs_tol=1e-9)


@pytest.mark.parametrize("cov1u,theta,n,a", [(0, 100, 1000, 5.0), (37, 1000, 5000, 12.3),
                                             (123456, 1 << 20, 1 << 20, 16.9)])
def test_upper_bound_is_the_root_of_the_lower_tail(orc, cov1u, theta, n, a):
    """x = sigma_u theta / n satisfies cov1u = x - sqrt(2 a x), x >= cov1u."""
    x = opim.upper(cov1u, theta, n, a) * theta / n
    assert x >= cov1u
    assert math.isclose(x - math.sqrt(2 * a * x), cov1u, rel_tol=1e-12, abs_tol=1e-9)


@pytest.mark.parametrize("n,k,eps,delta", [(1 << 20, 1000, 0.01, 2.0 ** -20),
                                           (1 << 20, 100, 0.1, 2.0 ** -20), (5000, 20, 0.2, 0.01),
                                           (100, 2, 0.3, 0.05)])
def test_theta_max_spends_the_final_budget(orc, n, k, eps, delta):
    """With OPT >= k, L = theta_max k samples per unit of OPT must make the
    lower tail of the optimal set and the union over C(n,k) bad sets of the
    upper tail each equal delta/6 (IMM's derivation with ln(6/delta) in place
    of ln(2 n^l)).  ln C(n,k) from the exact integer binomial."""
    c = opim.constants(n, k, eps, delta)
    L = c["theta_max"] * k
    q = 1 - 1 / math.e
    budget = math.log(6 / delta)
    e1 = math.sqrt(2 * n * budget / L)
    assert 0 < q * e1 < eps
    assert math.isclose(math.log(math.comb(n, k)) - (eps - q * e1) ** 2 * L / (2 * q * n),
                        -budget, rel_tol=1e-9)
    # theta_0 = ceil(theta_max eps^2 k / n), exactly
    t0 = Fraction(c["theta_max"]) * Fraction(eps) ** 2 * k / n
    assert c["theta0"] - 1 < t0 <= c["theta0"]
    # rounds: i_max = ceil(log2(theta_max / theta_0)) >= 1, and the budget a
    imax = max(1, math.ceil(math.log2(c["theta_max"] / c["theta0"])))
    assert c["rounds"] == imax
    assert math.isclose(3 * imax * math.exp(-c["a"]), delta, rel_tol=1e-12)


def test_round_cap(orc):
    c = opim.constants(1 << 20, 1000, 0.01, 2.0 ** -20, 1 << 20)
    t0 = c["theta0"]
    assert (t0 << (c["rounds"] - 1)) <= 1 << 20 < (t0 << c["rounds"])
    assert opim.constants(1 << 20, 1000, 0.01, 2.0 ** -20, 1)["rounds"] == 1


def _tiny(n, m, gseed, p):
    return inputs.random_graph(n, m, gseed, p)


@pytest.mark.parametrize("gseed", [1, 2, 3, 4])
def test_opim_rounds_halves_and_scores(orc, gseed):
    """The halves use disjoint ids (R2 from 2^31), the rounds double theta, cov2
    is the number of R2 sets holding a seed, cov1u bounds the optimal k-set's
    coverage of R1 (brute force), and alpha = sigma_l / sigma_u <= 1."""
    g = _tiny(9, 20, gseed, "0.4")
    k = 2
    r = opim.opim(g, orc.IC, k, 0.3, 0.05, 11)
    for i, th in enumerate(r.thetas):
        assert th == r.thetas[0] << i
    th = r.thetas[-1]
    p1 = orc.sample(orc.IC, g, 11, 0, th)
    p2 = orc.sample(orc.IC, g, 11, opim.R2_FIRST, th)
    S = set(int(v) for v in r.seeds)
    hits = sum(1 for i in range(th) if S & set(p2.set(i).tolist()))
    assert hits == r.cov2[-1]
    sub1 = brute.covering_subsets(g.n, [p1.set(i).tolist() for i in range(th)])
    assert r.cov1[-1] == brute.coverage(sub1, sorted(S))
    assert r.cov1u[-1] >= brute.optimal_cover(sub1, k)
    assert all(0 < a <= 1 for a in r.alphas if a > 0)


@pytest.mark.parametrize("gseed,p", [(1, "0.5"), (2, "0.6"), (5, "0.4"), (7, "0.7")])
def test_opim_guarantee_holds_on_exact_spreads(orc, gseed, p):
    """The instance-wise guarantee is a lower bound on sigma(S) / OPT: sigma
    exactly by enumerating every live-edge world of an 11- to 12-edge graph,
    OPT by enumerating every k-subset (holds with probability >= 1 - delta)."""
    g = _tiny(8, 12, gseed, p)
    k = 2
    for rg in (None, (3, 5, 1, 0.2)):
        r = opim.opim(g, orc.IC, k, 0.2, 0.01, 3, randgreedi=rg)
        alpha = r.alphas[-1]
        sigma = brute.ic_spread_exact(g, [int(v) for v in r.seeds])
        opt = max(brute.ic_spread_exact(g, list(Sx)) for Sx in itertools.combinations(range(g.n), k))
        assert float(sigma) >= alpha * float(opt)
        assert r.sigma_l <= float(sigma) <= float(opt) <= r.sigma_u
