"""The seeded workload generators: determinism and the stated parameter ranges."""
import numpy as np

from paper_2408_10982_gb300 import inputs


def test_batched_queries_ranges_and_determinism():
    a = inputs.batched_queries(256, 42)
    b = inputs.batched_queries(256, 42)
    assert [(q.graph, q.model, q.k, q.theta, q.seed) for q in a] == \
           [(q.graph, q.model, q.k, q.theta, q.seed) for q in b]
    assert len(a) == 256
    for q in a:
        assert q.graph in {f"rmat{s}" for s in inputs.BATCH_SCALES}
        assert q.model in (0, 1)
        assert 5 <= q.k <= 100
        assert (1 << 14) <= q.theta <= (1 << 20)
    assert len({q.seed for q in a}) == 256
    models = np.array([q.model for q in a])
    assert 0.35 < models.mean() < 0.65          # IC or LT with probability 1/2 each
    assert inputs.batched_queries(256, 43)[0].seed != a[0].seed


def test_served_trace_arrivals_and_orkut_share():
    t = inputs.served_trace(4000, 42, rate_per_s=200.0, orkut_frac=0.05)
    arr = np.array([q.arrival_s for q in t])
    assert np.all(np.diff(arr) > 0)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0   # exponential gaps, mean 5 ms
    ork = [q for q in t if q.graph == "orkut"]
    assert 0.03 < len(ork) / len(t) < 0.07
    for q in ork:
        assert q.model == 0 and (1 << 6) <= q.theta <= (1 << 10)
    assert all(q.graph != "orkut" for q in inputs.served_trace(500, 42, orkut_frac=0.0))


def test_batched_graph_weights_are_inverse_indegree():
    g = inputs.batched_graph(12, 42)
    assert g.n == 1 << 12 and g.m == 16 << 12
    d = np.diff(g.in_off)
    per_v = np.repeat(np.where(d > 0, (1 << 32) // np.maximum(d, 1), 0), d)
    assert np.array_equal(g.w.astype(np.int64), np.minimum(per_v, (1 << 32) - 1))
    sums = np.add.reduceat(g.w.astype(np.int64), g.in_off[:-1][d > 0])
    assert np.all(sums <= 1 << 32)


def test_paper_weight_model_uniform_0_to_0_1():
    """Sec. 4.1: edge probabilities drawn U[0, 0.1].  IC keeps each draw; LT
    uses the same draws and scales a vertex's in-weights to sum to 1 only when
    they sum above 1."""
    g = inputs.rmat_graph(1 << 12, 1 << 16, 5, "u0.1")
    p = g.w.astype(np.float64) / 2 ** 32
    assert p.min() >= 0 and p.max() <= 0.1 + 1e-9
    assert abs(p.mean() - 0.05) < 0.002 and abs(np.median(p) - 0.05) < 0.003
    assert np.array_equal(inputs.rmat_graph(1 << 12, 1 << 16, 5, "u0.1").w, g.w)
    lt = inputs.rmat_graph(1 << 12, 1 << 16, 5, "lt-u0.1")
    assert np.array_equal(lt.in_off, g.in_off) and np.array_equal(lt.in_src, g.in_src)
    d = np.diff(g.in_off)
    owner = np.repeat(np.arange(g.n), d)
    raw = np.bincount(owner, weights=p, minlength=g.n)
    sums = np.bincount(owner, weights=lt.w.astype(np.float64), minlength=g.n)
    assert np.all(sums <= 2 ** 32)
    small = raw <= 1.0                                  # kept: within quantisation
    assert np.all(np.abs(lt.w.astype(np.float64) - g.w.astype(np.float64))[small[owner]] <= 1.0)
    big = raw > 1.0                                     # scaled to sum 1
    assert big.any() and np.all(np.abs(sums[big] / 2 ** 32 - 1.0) < 1e-6)
