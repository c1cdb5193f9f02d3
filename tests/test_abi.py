"""The C-ABI library loads, exports every symbol its headers declare, and rejects
bad arguments before touching a GPU (CPU only)."""
import glob
import os
import re

import numpy as np
import pytest

import paper_2112_10603_b300 as fvv
from paper_2112_10603_b300 import build as fvv_build
from synth import weights

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fvv_build.build()
    return fvv.lib()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(fvv_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_blob_size_matches_generator(lib):
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_interp_create(np.zeros(weights.n_floats() - 1, np.float32), 64, 64)
    assert e.value.code == fvv.FVV_ESHAPE
    assert str(weights.n_floats()) in str(e.value)


@pytest.mark.parametrize("H,W,opts,code", [
    (8, 64, {}, fvv.FVV_ESHAPE),
    (64, 9000, {}, fvv.FVV_ESHAPE),
    (72, 64, {"pad_mode": fvv.FVV_PAD_CIRCULAR}, fvv.FVV_ESHAPE),
    (64, 64, {"precision": 7}, fvv.FVV_EINVAL),
    (64, 64, {"max_views": 0}, fvv.FVV_ESHAPE),
])
def test_create_rejects_bad_arguments(lib, H, W, opts, code):
    blob = np.zeros(weights.n_floats(), np.float32)
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_interp_create(blob, H, W, fvv.fvv_default_opts(**opts))
    assert e.value.code == code


def test_default_opts(lib):
    o = fvv.fvv_default_opts()
    assert (o.precision, o.pad_mode, o.t_mode, o.max_views, o.max_cams) == (0, 0, 0, 16, 2)


def test_noalloc_source_allocates_nothing():
    """The allocation-free entry point's source calls no device allocator (its only
    scratch is a file-scope __device__ array)."""
    src = open(os.path.join(ROOT, "paper_2112_10603_b300", "csrc", "noalloc.cu")).read()
    code = re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", src, flags=re.S))
    for banned in ("cudaMalloc", "cudaFree", "cuMemAlloc", "cuMemFree", "dalloc", "torch", "new ", "malloc("):
        assert banned not in code, banned
    assert re.search(r"static\s+__device__\s+__align__\(256\)\s+float\s+g_noalloc_w\[", code)
    assert "cudaGetSymbolAddress" in code


def test_lap_loss_workspace_plan(lib):
    """The loss's workspace (pyramid levels 2-5 + block sums) grows with the views and
    is 0 for sizes the call rejects; no GPU needed."""
    one = fvv.fvv_lap_loss_workspace(1, 1080, 1920)
    seven = fvv.fvv_lap_loss_workspace(7, 1080, 1920)
    # levels 2..5 hold about a third of a full-size image per view
    assert 0.3 < one / (1080 * 1920 * 12) < 0.4
    assert 6.9 < seven / one < 7.1
    assert fvv.fvv_lap_loss_workspace(0, 8, 8) == 0 and fvv.fvv_lap_loss_workspace(1, 1, 8) == 0
