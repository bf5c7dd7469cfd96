"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/knnm.h declares; the Python binding covers exactly those.  No
compute call is made here (no GPU needed)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "knnm.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(knnm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1908_00814_gb300 import build
    path = build.build()
    return ctypes.CDLL(str(path))


def test_header_declares_the_merge_calls():
    names = declared_functions()
    for must in ("knnm_merge_symmetric", "knnm_merge_joint", "knnm_build", "knnm_step_init",
                 "knnm_step_sample", "knnm_step_join", "knnm_step_final", "knnm_create",
                 "knnm_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_matches_header(built_lib):
    from paper_1908_00814_gb300 import knnm
    assert sorted(knnm.SIGNATURES) == declared_functions()


def test_library_targets_sm103a(built_lib):
    from paper_1908_00814_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_strerror_needs_no_gpu(built_lib):
    built_lib.knnm_strerror.restype = ctypes.c_char_p
    assert built_lib.knnm_strerror(-1) == b"invalid argument"
    built_lib.knnm_default_params.argtypes = [ctypes.c_void_p]
    from paper_1908_00814_gb300 import knnm
    p = knnm.Params()
    built_lib.knnm_default_params(ctypes.byref(p))
    assert p.k == 20 and abs(p.sample_rate - 0.5) < 1e-7 and p.max_iters == 10


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1908_00814_gb300 import knnm
    monkeypatch.setattr(knnm, "_LIB_PATH", tmp_path / "missing.so")
    monkeypatch.setattr(knnm, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        knnm.lib()


@pytest.mark.parametrize("K", [1, 7, 10, 20, 31, 32])
@pytest.mark.parametrize("r,rho", [(0.5, 0.5), (0.3, 0.25), (0.0, 1.0), (1.0, 0.1)])
def test_list_widths_match_the_oracle(built_lib, orc, K, r, rho):
    """The sizes the library derives (no GPU call): K_keep = floor(r K) as the
    oracle's Divide keeps, Kr = K - K_keep, s = max(1, floor(rho K)); a build
    (J-Merge of an empty graph) keeps all K."""
    from paper_1908_00814_gb300 import knnm
    p = knnm.params(k=K, keep_ratio=r, sample_rate=rho)
    kk, kr, s = knnm.list_widths(p, knnm.SYMMETRIC, 100)
    assert kk == orc.keep_count(K, r) and kr == K - kk
    assert s == min(K, orc.sample_count(K, rho))
    assert knnm.list_widths(p, knnm.JOINT, 0)[:2] == (K, 0)
    with pytest.raises(knnm.KnnmError):
        knnm.list_widths(knnm.params(k=33), knnm.SYMMETRIC, 100)


def test_caller_output_buffers_are_checked():
    """Output buffers passed by the caller (pinned host memory, say) come back
    as given when they are contiguous [n, k] int32 / float32, and are refused
    before any library call otherwise."""
    import numpy as np
    import torch
    from paper_1908_00814_gb300 import knnm
    outputs = knnm.Context._outputs
    n, k = 7, 5
    for make in (lambda s, dt: np.zeros(s, dt), lambda s, dt: torch.zeros(s, dtype=getattr(torch, dt))):
        ids, dists = make((n, k), "int32"), make((n, k), "float32")
        got = outputs(None, None, n, k, (ids, dists))
        assert got[0] is ids and got[1] is dists
        with pytest.raises(ValueError):
            outputs(None, None, n, k, (make((n, k), "int64"), dists))
        with pytest.raises(ValueError):
            outputs(None, None, n, k, (ids, make((n, k + 1), "float32")))
        with pytest.raises(ValueError):
            outputs(None, None, n, k, (make((k, n), "int32").T, dists))
