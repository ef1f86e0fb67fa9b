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


def _header_constants():
    """Every enum value and numeric #define named FBS_* in include/*.h."""
    out = {}
    for fname in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fname.endswith(".h"):
            continue
        text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", fname)).read(), flags=re.S)
        for name, expr in re.findall(r"#define\s+(FBS_[A-Z0-9_]+)\s+([^\n]+)", text):
            expr = re.sub(r"(\d+)[uUlL]+\b", r"\1", expr.strip())
            if re.fullmatch(r"[\d\s()*+<-]+", expr):
                out[name] = eval(expr)
        for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
            for name, val in re.findall(r"(FBS_[A-Z0-9_]+)\s*=\s*(\d+)", body):
                out[name] = int(val)
    return out


def test_python_constants_match_the_header(fbs):
    consts = _header_constants()
    assert consts["FBS_NOALLOC_MAX_COST_BYTES"] == 32 * 1024 * 1024
    assert consts["FBS_ERR_TIMEOUT"] == 4 and consts["FBS_PREC_F16"] == 2
    for name, val in consts.items():
        assert hasattr(fbs, name), f"{name} declared in include/ but not bound"
        assert getattr(fbs, name) == val, f"{name}: binding {getattr(fbs, name)} != header {val}"


def test_noalloc_limit_formula_matches_the_header_examples(fbs):
    """The documented limit H*W*(4*round_up(D,4)+20) bytes: 640x480 fits up to
    D=20 and 320x240 up to D=104, the largest D of each that fits."""
    cap = fbs.FBS_NOALLOC_MAX_COST_BYTES

    def need(H, W, D):
        n = 2 * H * W
        r = lambda b: (b + 255) // 256 * 256
        return r(2 * n) + r(4 * n) + r(4 * n) + 4 * H * W * ((D + 3) // 4 * 4)

    def largest_D(H, W):
        return max(D for D in range(1, 1025) if need(H, W, D) <= cap)

    assert largest_D(480, 640) == 20
    assert largest_D(240, 320) == 104
    for H, W, D in [(480, 640, 20), (240, 320, 104), (100, 200, 64)]:
        assert abs(need(H, W, D) - H * W * (4 * ((D + 3) // 4 * 4) + 20)) < 4 * 256


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
