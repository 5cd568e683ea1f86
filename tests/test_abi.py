"""The C-ABI library builds, loads and exports every entry point include/im.h declares.

No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "im.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(im_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2408_10982_gb300 import build
    return build.build_library()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("im_sample_rrr", "im_max_k_cover", "im_graph_create", "im_pool_create",
                 "im_pool_export", "im_status_str"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    from paper_2408_10982_gb300 import im
    assert im.status_str(0) == "ok"
    assert "capacity" in im.status_str(im.IM_ERR_CAPACITY)


# --- host-side behaviour of the boundary (no device work) ---------------------

def _no_gpu():
    try:
        import torch
        return not torch.cuda.is_available()
    except ImportError:
        return True


def test_tuning_knobs_defaults_values_and_rejections(libpath):
    """The knob values include/im.h documents: defaults 1, 0, 0, 2, 0, 0, 8; every
    allowed value is stored; anything else is IM_ERR_INVALID_ARG and leaves
    the knob unchanged."""
    from paper_2408_10982_gb300 import im
    allowed = {im.IM_TUNE_LT_GROUP: [1, 8, 16, 32],
               im.IM_TUNE_RG_CLUSTER: [-1, 0, 1, 2, 4, 8],
               im.IM_TUNE_INDEX_REPLICAS: [0, 1, 2, 4, 8],
               im.IM_TUNE_RG_EVALS: [1, 2, 4, 8],
               im.IM_TUNE_GREEDY_EVALS: [0, 1, 2, 4, 8, 16, 32],
               im.IM_TUNE_LT_CACHE: [0, 1, 2],
               im.IM_TUNE_GREEDY_HOT: [0, 4, 8, 12, 16]}
    defaults = {im.IM_TUNE_LT_GROUP: 1, im.IM_TUNE_RG_CLUSTER: 0,
                im.IM_TUNE_INDEX_REPLICAS: 0, im.IM_TUNE_RG_EVALS: 2,
                im.IM_TUNE_GREEDY_EVALS: 0, im.IM_TUNE_LT_CACHE: 0,
                im.IM_TUNE_GREEDY_HOT: 8}
    before = {k: im.im_tune_get(k) for k in allowed}
    try:
        for k in allowed:
            im.im_tune_set(k, defaults[k])
        for k, vals in allowed.items():
            for v in vals:
                im.im_tune_set(k, v)
                assert im.im_tune_get(k) == v
            keep = im.im_tune_get(k)
            for bad in (0 if k not in (im.IM_TUNE_RG_CLUSTER, im.IM_TUNE_LT_CACHE,
                                       im.IM_TUNE_GREEDY_HOT) else 3, 3, 17, 64, -2, 1 << 40):
                if bad in vals:
                    continue
                with pytest.raises(im.ImError) as e:
                    im.im_tune_set(k, bad)
                assert e.value.status == im.IM_ERR_INVALID_ARG
                assert im.im_tune_get(k) == keep
        for bad_knob in (-1, 7, 99):
            with pytest.raises(im.ImError):
                im.im_tune_set(bad_knob, 1)
            with pytest.raises(im.ImError):
                im.im_tune_get(bad_knob)
    finally:
        for k, v in before.items():
            im.im_tune_set(k, v)
    assert before == defaults


def test_invalid_arguments_rejected_before_any_device_work(libpath):
    """Argument checks are host logic: they answer IM_ERR_INVALID_ARG, with a
    message, whether or not a GPU is present."""
    from paper_2408_10982_gb300 import im
    import numpy as np
    off = np.array([0, 1], np.int64)
    src = np.array([0], np.int32)
    w = np.array([1], np.uint32)
    for args in ((off, src, w, 0, 1), (off, src, w, 1, -1), (off, src, w, 1 << 31, 1),
                 (off, None, w, 1, 1), (off, src, None, 1, 1)):
        with pytest.raises(im.ImError) as e:
            im.im_graph_create(*args)
        assert e.value.status == im.IM_ERR_INVALID_ARG
        assert "im_graph_create" in str(e.value)
    with pytest.raises(im.ImError) as e:
        im.im_pool_create(None, 10, 10)
    assert e.value.status == im.IM_ERR_INVALID_ARG
    # server options: a heavy lane needs a second worker; bounds are positive
    for kw in (dict(workers=1, heavy_members=1000), dict(workers=2, heavy_members=-1),
               dict(workers=0), dict(workers=17), dict(max_batch=0), dict(mem_budget=0)):
        with pytest.raises(im.ImError) as e:
            im.im_server_create(**kw)
        assert e.value.status == im.IM_ERR_INVALID_ARG


@pytest.mark.skipif(not _no_gpu(), reason="checks the answer on a machine without a GPU")
def test_device_calls_report_unsupported_without_gpu(libpath):
    from paper_2408_10982_gb300 import im
    for call in (im.im_device_info, im.im_trim_memory):
        with pytest.raises(im.ImError) as e:
            call()
        assert e.value.status == im.IM_ERR_UNSUPPORTED
