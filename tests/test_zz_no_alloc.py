"""The allocation-free layer call (fvv_layer_noalloc) against the regular one.

fvv_layer_noalloc serves callers that may not allocate device memory (a host
application with a fixed device-memory budget, a real-time loop that cannot risk
an allocation's synchronisation, a plug-in inside another framework's memory
pool).  It keeps its only scratch — the repacked weights — in a fixed device
array shared by all calls.  This test checks, through the C ABI, that its output
matches fvv_interp_layer on an FP32 handle (the existing entry point) within the
FP32 tolerance of the other tests, on consecutive calls with different layers
(so the shared array's previous contents cannot leak into the next call).

The file is named so that pytest collects it last; it runs alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

import paper_2112_10603_b300 as fvv
from synth import weights

pytestmark = pytest.mark.gpu

TOL = 1e-4
# conv s1 (256 ch), conv s2, convT, ContextNet's 3-channel first layer, output conv
LAYERS = ["vib0.m0", "vib0.c1", "vib1.t0", "ctx.c0", "ref.out", "ref.d0"]


def test_noalloc_layer_matches_interp_layer():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    blob = weights.he_init(0)
    manifest = {m[0]: (i, m) for i, m in enumerate(weights.manifest())}
    views = weights.layer_views(blob)
    it = fvv.Interpolator(blob, 64, 64, precision=fvv.FVV_FP32, max_views=1)
    rng = np.random.default_rng(7)
    for rep in range(2):                      # two rounds: every call follows another layer's call
        for name in LAYERS:
            li, (_, kind, ci, co, stride, _) = manifest[name]
            H, W = (10, 18) if kind == "convT" else (22, 36)
            n, cs = 2, ci + 5
            x = torch.from_numpy(rng.standard_normal((n, H, W, cs)).astype(np.float32)).cuda()
            Ho, Wo = (2 * H, 2 * W) if kind == "convT" else ((H - 1) // stride + 1, (W - 1) // stride + 1)
            w, b = views[name]
            wd = torch.from_numpy(np.ascontiguousarray(w)).cuda()
            bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
            ref = torch.zeros((n, Ho, Wo, co), device="cuda")
            got = torch.full((n, Ho, Wo, co + 2), -3.0, device="cuda")
            fvv.fvv_interp_layer(it.h, li, x, cs, 5, n, H, W, ref, co, 0, True)
            fvv.fvv_layer_noalloc(li, wd, bd, x, cs, 5, n, H, W, got, co + 2, 1)
            torch.cuda.synchronize()
            g = got.cpu().numpy()
            r = ref.cpu().numpy()
            assert (g[..., 0] == -3).all() and (g[..., co + 1] == -3).all(), "wrote outside its channel slot"
            scale = max(1.0, float(np.abs(r).max()))
            err = float(np.abs(g[..., 1:1 + co] - r).max())
            assert err <= TOL * scale, (rep, name, err)
    fvv.fvv_interp_status(it.h)
    it.close()


def test_noalloc_rejects_bad_arguments():
    import torch
    x = torch.zeros(16, device="cuda")
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_layer_noalloc(99, x, x, x, 8, 0, 1, 4, 4, x, 8, 0)
    assert e.value.code == fvv.FVV_EINVAL
    with pytest.raises(fvv.FvvError) as e:   # stride-2 layer with an odd size
        fvv.fvv_layer_noalloc(0, x, x, x, 16, 0, 1, 5, 4, x, 128, 0)
    assert e.value.code == fvv.FVV_ESHAPE
