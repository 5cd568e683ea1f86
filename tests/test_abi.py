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
