"""Host-side checks of the C ABI: the library builds, loads and exports every
symbol the header declares; calls with a NULL context fail cleanly."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(fbs_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def fbs():
    from paper_1807_02044_gb300 import build as b
    b.build()
    import paper_1807_02044_gb300 as m
    return m


def test_header_declares_the_path(fbs):
    names = _declared_functions()
    for required in ["fbs_create", "fbs_destroy", "fbs_compute_disparity", "fbs_cost_volume", "fbs_aggregate"]:
        assert required in names


def test_every_declared_symbol_is_exported_and_bound(fbs):
    lib = ctypes.CDLL(fbs.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert name in fbs.SIGNATURES, f"{name} has no binding"


def test_null_context_calls_fail_cleanly(fbs):
    lib = fbs.lib()
    assert lib.fbs_destroy(None) == fbs.FBS_OK
    assert lib.fbs_sync(None) == fbs.FBS_ERR_INVALID_ARG
    assert lib.fbs_last_error(None) == b"null context"
    assert lib.fbs_compute_disparity(None, None, None, 1, 1, 1, 1, 0, 1.0, 1.0, 0.0, None, None, None) == \
        fbs.FBS_ERR_INVALID_ARG
    assert lib.fbs_create(None, None, 0) == fbs.FBS_ERR_INVALID_ARG


def test_default_options(fbs):
    o = fbs.fbs_default_options()
    assert (o.cost, o.prec, o.fused, o.workspace_cap) == (0, 0, 0, 0)


def test_create_without_gpu_reports_cuda_error(fbs):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fbs.FBSError) as ei:
        fbs.fbs_create(None, 0)
    assert ei.value.status in (fbs.FBS_ERR_CUDA, fbs.FBS_ERR_INVALID_ARG)
