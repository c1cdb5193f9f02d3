"""The allocation-free layer call (fvv_layer_noalloc) against the regular one and the oracle.

fvv_layer_noalloc serves callers that may not allocate device memory (a host
application with a fixed device-memory budget, a real-time loop that cannot risk
an allocation's synchronisation, a plug-in inside another framework's memory
pool).  It keeps its only scratch -- the repacked weights -- in a fixed device
array shared by all calls.  Through the C ABI this test checks, on two rounds of
consecutive calls with different layers (so the shared array's previous contents
cannot leak into the next call):

* its output matches fvv_interp_layer on an FP32 handle (the existing entry point)
  within the FP32 tolerance of the other tests;
* its output matches the oracle's conv / transposed conv (FP64) within that same
  tolerance;
* the second round of calls leaves the device's free memory unchanged (the first
  call on a device loads the module and with it the array; later calls allocate
  nothing).

The file is named so that pytest collects it last; it runs alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

import oracle
import paper_2112_10603_b300 as fvv
from synth import weights

pytestmark = pytest.mark.gpu

TOL = 1e-4
# conv s1 (256 ch), conv s2, convT, ContextNet's 3-channel first layer, output conv
LAYERS = ["vib0.m0", "vib0.c1", "vib1.t0", "ctx.c0", "ref.out", "ref.d0"]


def _oracle_layer(kind, x, w, b, stride, relu):
    if kind == "conv":
        return oracle.conv3x3(x, w, b, stride=stride, relu=relu)
    return oracle.conv_transpose4x4(x, w, b, relu=relu)


def test_noalloc_layer_matches_interp_layer_and_oracle():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    blob = weights.he_init(0)
    manifest = {m[0]: (i, m) for i, m in enumerate(weights.manifest())}
    views = weights.layer_views(blob)
    it = fvv.Interpolator(blob, 64, 64, precision=fvv.FVV_FP32, max_views=1)
    rng = np.random.default_rng(7)
    # every buffer is allocated before the first call, so that the free-memory check
    # below sees only what the calls themselves allocate
    cases = []
    for name in LAYERS:
        li, (_, kind, ci, co, stride, relu) = manifest[name]
        H, W = (10, 18) if kind == "convT" else (22, 36)
        n, cs = 2, ci + 5
        xh = rng.standard_normal((n, H, W, cs)).astype(np.float32)
        Ho, Wo = (2 * H, 2 * W) if kind == "convT" else ((H - 1) // stride + 1, (W - 1) // stride + 1)
        w, b = views[name]
        ref_o = np.stack([_oracle_layer(kind, xh[i, ..., 5:5 + ci], w, b, stride, relu) for i in range(n)])
        cases.append(dict(
            name=name, li=li, co=co, n=n, H=H, W=W, cs=cs, ref_o=ref_o,
            x=torch.from_numpy(xh).cuda(),
            w=torch.from_numpy(np.ascontiguousarray(w)).cuda(),
            b=torch.from_numpy(np.ascontiguousarray(b)).cuda(),
            ref=torch.zeros((n, Ho, Wo, co), device="cuda"),
            got=torch.empty((n, Ho, Wo, co + 2), device="cuda")))
    torch.cuda.synchronize()
    free_after = []
    for rep in range(2):                      # two rounds: every call follows another layer's call
        for c in cases:
            c["got"].fill_(-3.0)
            fvv.fvv_interp_layer(it.h, c["li"], c["x"], c["cs"], 5, c["n"], c["H"], c["W"], c["ref"], c["co"], 0,
                                 True)
            fvv.fvv_layer_noalloc(c["li"], c["w"], c["b"], c["x"], c["cs"], 5, c["n"], c["H"], c["W"], c["got"],
                                  c["co"] + 2, 1)
            torch.cuda.synchronize()
            co = c["co"]
            g = c["got"].cpu().numpy()
            r = c["ref"].cpu().numpy()
            assert (g[..., 0] == -3).all() and (g[..., co + 1] == -3).all(), "wrote outside its channel slot"
            scale = max(1.0, float(np.abs(c["ref_o"]).max()))
            err = float(np.abs(g[..., 1:1 + co] - r).max())
            assert err <= TOL * scale, (rep, c["name"], "vs fvv_interp_layer", err)
            err_o = float(np.abs(g[..., 1:1 + co] - c["ref_o"]).max())
            assert err_o <= TOL * scale, (rep, c["name"], "vs oracle", err_o)
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
    # a device allocation takes at least a 2 MiB page; the second round made none
    assert abs(free_after[1] - free_after[0]) < (1 << 20), free_after
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
