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
