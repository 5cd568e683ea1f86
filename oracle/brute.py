"""Brute force on tiny inputs -- TEST INFRASTRUCTURE ONLY.

Exact answers computed straight from the definitions, used to pin the oracle:
  - inclusion probabilities P(v in RRR(root)) by enumerating every live-edge
    world (IC: each edge live independently, Def. 3; LT: each vertex keeps at
    most one in-edge, chosen with probability equal to its weight, Sec. 2);
  - the optimal max-k-cover by enumerating all k-subsets (Sec. 3.2);
  - greedy by recomputing every marginal gain C(S + v) - C(S) from scratch
    with Python sets.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

TWO32 = 1 << 32


def _reverse_reach(n, in_off, in_src, live, root):
    seen = {root}
    stack = [root]
    while stack:
        v = stack.pop()
        for e in range(int(in_off[v]), int(in_off[v + 1])):
            if live[e]:
                u = int(in_src[e])
                if u not in seen:
                    seen.add(u)
                    stack.append(u)
    return seen


def ic_inclusion_exact(graph, root: int) -> list[Fraction]:
    """P(v in RRR(root)) under IC with p_e = w[e] / 2^32, for every v."""
    n, m = graph.n, graph.m
    p = [Fraction(int(x), TWO32) for x in graph.w]
    out = [Fraction(0)] * n
    for mask in range(1 << m):
        live = [(mask >> e) & 1 for e in range(m)]
        prob = Fraction(1)
        for e in range(m):
            prob *= p[e] if live[e] else 1 - p[e]
        if prob == 0:
            continue
        for v in _reverse_reach(n, graph.in_off, graph.in_src, live, root):
            out[v] += prob
    return out


def lt_inclusion_exact(graph, root: int) -> list[Fraction]:
    """P(v in RRR(root)) under LT: vertex v keeps in-edge e w.p. w[e]/2^32."""
    n = graph.n
    options = []
    for v in range(n):
        b, e = int(graph.in_off[v]), int(graph.in_off[v + 1])
        opts = [(None, Fraction(TWO32 - sum(int(graph.w[x]) for x in range(b, e)), TWO32))]
        opts += [(x, Fraction(int(graph.w[x]), TWO32)) for x in range(b, e)]
        options.append(opts)
    out = [Fraction(0)] * n
    for choice in itertools.product(*options):
        prob = Fraction(1)
        for _, pr in choice:
            prob *= pr
        if prob == 0:
            continue
        seen = [root]
        cur = root
        while True:
            e = choice[cur][0]
            if e is None:
                break
            u = int(graph.in_src[e])
            if u in seen:
                break
            seen.append(u)
            cur = u
        for v in seen:
            out[v] += prob
    return out


def coverage(subsets: list[set], chosen) -> int:
    u = set()
    for v in chosen:
        u |= subsets[v]
    return len(u)


def optimal_cover(subsets: list[set], k: int, cand=None) -> int:
    """max |union of S(v), v in X| over |X| <= k (monotone, so |X| = min(k, |cand|))."""
    cand = list(range(len(subsets))) if cand is None else list(cand)
    kk = min(k, len(cand))
    best = 0
    for combo in itertools.combinations(cand, kk):
        best = max(best, coverage(subsets, combo))
    return best


def greedy_definition(subsets: list[set], k: int, cand=None):
    """Greedy max-k-cover recomputing each marginal gain from scratch."""
    cand = sorted(range(len(subsets))) if cand is None else sorted(cand)
    covered: set = set()
    seeds, gains = [], []
    for _ in range(k):
        best, best_gain = None, 0
        for v in cand:
            g = len(subsets[v] - covered)
            if g > best_gain:
                best, best_gain = v, g
        if best is None:
            break
        seeds.append(best)
        gains.append(best_gain)
        covered |= subsets[best]
    return seeds, gains, len(covered)


def covering_subsets(n: int, sets: list) -> list[set]:
    """S(v) = {i : v in R(i)} from a list of RRR sets."""
    out = [set() for _ in range(n)]
    for i, r in enumerate(sets):
        for v in r:
            out[int(v)].add(i)
    return out


def _forward_reach(n, in_off, in_src, live, seeds):
    out = [[] for _ in range(n)]
    for v in range(n):
        for e in range(int(in_off[v]), int(in_off[v + 1])):
            if live[e]:
                out[int(in_src[e])].append(v)
    seen = set(int(s) for s in seeds)
    stack = list(seen)
    while stack:
        u = stack.pop()
        for v in out[u]:
            if v not in seen:
                seen.add(v)
                stack.append(v)
    return seen


def ic_spread_exact(graph, seeds) -> Fraction:
    """sigma(S) = E |vertices reachable from S| over every IC live-edge world."""
    m = graph.m
    p = [Fraction(int(x), TWO32) for x in graph.w]
    total = Fraction(0)
    for mask in range(1 << m):
        live = [(mask >> e) & 1 for e in range(m)]
        prob = Fraction(1)
        for e in range(m):
            prob *= p[e] if live[e] else 1 - p[e]
        if prob:
            total += prob * len(_forward_reach(graph.n, graph.in_off, graph.in_src, live, seeds))
    return total


def lt_spread_exact(graph, seeds) -> Fraction:
    """sigma(S) under LT: each vertex keeps at most one in-edge (w / 2^32 each)."""
    n, m = graph.n, graph.m
    options = []
    for v in range(n):
        b, e = int(graph.in_off[v]), int(graph.in_off[v + 1])
        opts = [(None, Fraction(TWO32 - sum(int(graph.w[x]) for x in range(b, e)), TWO32))]
        opts += [(x, Fraction(int(graph.w[x]), TWO32)) for x in range(b, e)]
        options.append(opts)
    total = Fraction(0)
    for choice in itertools.product(*options):
        prob = Fraction(1)
        live = [0] * m
        for e, pr in choice:
            prob *= pr
            if e is not None:
                live[e] = 1
        if prob:
            total += prob * len(_forward_reach(n, graph.in_off, graph.in_src, live, seeds))
    return total
