"""The allocation-free greedy entry point (im_max_k_cover_noalloc).

It serves callers that cannot let a library allocate device memory (a
framework's caching allocator owns the GPU, a request loop cannot pay for
cudaMalloc).  It runs the standard greedy on arrays the caller owns with a
fixed static scratch array inside the library, so it must give exactly what
im_max_k_cover gives -- on consecutive calls, since the scratch is reused.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2408_10982_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_10982_gb300 import build, im
    build.build_library()
    return torch, im


def _device_instance(torch, im, g, model, theta, seed):
    G = im.Graph(g)
    P = im.Pool(G, theta, theta * min(g.n, 512))
    P.sample(model, seed, 0, theta)
    set_off, members = P.export()
    vtx_off, set_ids = P.index()
    dev = [torch.from_numpy(a).cuda() for a in (set_off, members, vtx_off, set_ids)]
    return G, P, dev


@pytest.mark.parametrize("k", [16, 100])
def test_noalloc_matches_pool_cover_on_consecutive_calls(env, k):
    torch, im = env
    for g, model, theta in ((inputs.rmat_graph(1 << 14, 1 << 18, 42, "lt"), im.IM_LT, 60000),
                            (inputs.graph_small_ic(), im.IM_IC, 16384)):
        G, P, (so, mem, vo, si) = _device_instance(torch, im, g, model, theta, 11)
        ref = P.cover(k)
        for _ in range(2):
            seeds = torch.full((k,), -7, dtype=torch.int32, device="cuda")
            gains = torch.full((k,), -7, dtype=torch.int64, device="cuda")
            ns = torch.full((1,), -7, dtype=torch.int32, device="cuda")
            cov = torch.full((1,), -7, dtype=torch.int64, device="cuda")
            im.im_max_k_cover_noalloc(so, mem, vo, si, g.n, theta, k, seeds, gains, ns, cov)
            m = int(ns.item())
            assert m == len(ref.seeds)
            assert seeds[:m].cpu().numpy().tolist() == ref.seeds.tolist()
            assert gains[:m].cpu().numpy().tolist() == ref.gains.tolist()
            assert int(cov.item()) == ref.coverage


def test_noalloc_rejects_instances_beyond_its_scratch(env):
    torch, im = env
    d = torch.zeros(8, dtype=torch.int64, device="cuda")
    i = torch.zeros(8, dtype=torch.int32, device="cuda")
    out64 = torch.zeros(4, dtype=torch.int64, device="cuda")
    out32 = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(im.ImError) as e:
        im.im_max_k_cover_noalloc(d, i, d, i, 20_000_000, 4, 4, out32, out64, out32, out64)
    assert e.value.status == im.IM_ERR_CAPACITY
    with pytest.raises(im.ImError) as e:
        host = np.zeros(4, np.int32)
        im.im_max_k_cover_noalloc(d, i, d, i, 4, 4, 4, host, out64, out32, out64)
    assert e.value.status == im.IM_ERR_INVALID_ARG


def _outputs(torch, k):
    return (torch.full((k,), -7, dtype=torch.int32, device="cuda"),
            torch.full((k,), -7, dtype=torch.int64, device="cuda"),
            torch.full((1,), -7, dtype=torch.int32, device="cuda"),
            torch.full((1,), -7, dtype=torch.int64, device="cuda"))


def _check_same(im, ref, k, args, n, theta, torch):
    seeds, gains, ns, cov = _outputs(torch, k)
    im.im_max_k_cover_noalloc(*args, n, theta, k, seeds, gains, ns, cov)
    m = int(ns.item())
    assert m == len(ref.seeds)
    assert seeds[:m].cpu().numpy().tolist() == ref.seeds.tolist()
    assert gains[:m].cpu().numpy().tolist() == ref.gains.tolist()
    assert int(cov.item()) == ref.coverage


def test_noalloc_empty_pool(env):
    """theta = 0: no sets, null member and set-id arrays; no seed, coverage 0,
    the same as the pool's own cover."""
    torch, im = env
    g = inputs.graph_small_ic()
    G = im.Graph(g)
    P = im.Pool(G, 16, 1024)
    ref = P.cover(8)
    so = torch.zeros(1, dtype=torch.int64, device="cuda")
    vo = torch.zeros(g.n + 1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        _check_same(im, ref, 8, (so, None, vo, None), g.n, 0, torch)
    assert len(ref.seeds) == 0 and ref.coverage == 0


# the largest n whose scratch fits with theta = 4096: 256 (control) + 32768
# (per-block maxima) + up256(4 n) + up256(theta / 8) <= 64 MiB
_THETA_EDGE = 4096
_N_EDGE = (64 * 2 ** 20 - 256 - 32768 - 512) // 4


def _big_sparse_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, size=m, dtype=np.int64)
    dst = rng.integers(0, n, size=m, dtype=np.int64)
    keep = src != dst
    key = np.unique(dst[keep] * n + src[keep])
    in_off, in_src = inputs.in_csr(n, (key % n).astype(np.int32), (key // n).astype(np.int32))
    w = np.full(in_src.size, 2 ** 31, np.uint32)            # IC p = 1/2
    return inputs.Graph(n, in_off, in_src, w)


def test_noalloc_at_the_edge_of_its_scratch(env):
    """An instance whose scratch need is exactly the 64 MiB array (n = 16,768,832,
    theta = 4096) equals the pool's cover on two calls in a row; 64 more
    vertices get IM_ERR_CAPACITY."""
    torch, im = env
    g = _big_sparse_graph(_N_EDGE, 1 << 23, 3)
    G, P, (so, mem, vo, si) = _device_instance(torch, im, g, im.IM_IC, _THETA_EDGE, 5)
    ref = P.cover(20)
    for _ in range(2):
        _check_same(im, ref, 20, (so, mem, vo, si), g.n, _THETA_EDGE, torch)
    seeds, gains, ns, cov = _outputs(torch, 20)
    vo_big = torch.zeros(_N_EDGE + 65, dtype=torch.int64, device="cuda")
    with pytest.raises(im.ImError) as e:
        im.im_max_k_cover_noalloc(so, mem, vo_big, si, _N_EDGE + 64, _THETA_EDGE, 20, seeds,
                                  gains, ns, cov)
    assert e.value.status == im.IM_ERR_CAPACITY


def test_noalloc_refuses_an_invalid_instance_then_runs_the_next(env):
    """A member id >= n or a decreasing offset is caught on the device before
    the greedy writes anything (IM_ERR_INVALID_ARG); the next valid call on the
    same scratch still equals the pool's cover."""
    torch, im = env
    g = inputs.graph_small_ic()
    G, P, (so, mem, vo, si) = _device_instance(torch, im, g, im.IM_IC, 4096, 9)
    ref = P.cover(16)
    bad_mem = mem.clone()
    bad_mem[7] = g.n
    bad_so = so.clone()
    bad_so[5] = bad_so[6] + 1
    seeds, gains, ns, cov = _outputs(torch, 16)
    for args in ((so, bad_mem, vo, si), (bad_so, mem, vo, si)):
        with pytest.raises(im.ImError) as e:
            im.im_max_k_cover_noalloc(*args, g.n, 4096, 16, seeds, gains, ns, cov)
        assert e.value.status == im.IM_ERR_INVALID_ARG
    _check_same(im, ref, 16, (so, mem, vo, si), g.n, 4096, torch)
