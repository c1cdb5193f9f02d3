"""Failure detection on the GPU without a GPU fault.

Every mbarrier wait in the tensor-core convolution is bounded; when one runs out the
kernel records an error code in the handle's device error word, tells the other warp
roles to stop, lets the copies it issued land, frees TMEM and returns, and
fvv_interp_status reports FVV_ETIMEOUT.  fvv_interp_inject_stall makes that happen
on purpose: it arms the next fvv_interp_layer call so that the kernel's MMA warp waits,
with a short limit, on a barrier that nothing signals.  For one layer of each kernel
form (per-tap, halo, grouped with resident weights, stride-2 pair halo, folded column
taps, per-phase transposed conv, RefineNet d3's own folded kernel) this test checks that

* the stalled call leaves its output untouched and the status is FVV_ETIMEOUT;
* the status word is cleared by reading it;
* the next call on the same handle runs normally and matches the oracle's conv of the
  same bf16-rounded operands (the bar of the per-layer tests).
"""
import numpy as np
import pytest

import oracle
import paper_2112_10603_b300 as fvv
from synth import weights
from tests.gpu_common import blob

pytestmark = pytest.mark.gpu

STALL_CYCLES = 2_000_000   # ~1 ms at the B300's clock

# layer, (H, W) of the input grid: each lands on a different producer / MMA branch
CASES = [
    ("vib0.m0", (3, 260)),   # 256-channel halo tiles
    ("vib0.c1", (6, 264)),   # per-tap stride-2 conv
    ("ref.e0a", (6, 264)),   # stride-2 pair halo, resident weights
    ("ref.e0b", (3, 260)),   # grouped halo stages, resident weights
    ("vib1.t1", (3, 370)),   # folded column taps (all-phase transposed conv)
    ("vib2.t0", (3, 131)),   # per-phase transposed conv
    ("ref.d3", (3, 131)),    # its own kernel (column taps folded into N = 192), bf16 output
]
BF16_OUT = {"ref.d3"}        # layers whose kernel takes bf16 output (the network's form)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    return torch


def _bf16_round(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


@pytest.mark.parametrize("name,grid", CASES)
def test_stalled_wait_reports_timeout_then_recovers(torch_cuda, name, grid):
    torch = torch_cuda
    names = [m[0] for m in weights.manifest()]
    li = names.index(name)
    _, kind, ci, co, stride, relu = weights.manifest()[li]
    H, W = grid
    n = 2
    cs = 16 if ci <= 16 else (32 if ci <= 32 else ci)   # narrow inputs: padded channel block
    rng = np.random.default_rng(900 + li)
    x = np.zeros((n, H, W, cs), np.float32)
    x[..., :ci] = rng.standard_normal((n, H, W, ci)) * 0.5
    x = _bf16_round(torch, x)
    wv, bv = weights.layer_views(blob())[name]
    wq = _bf16_round(torch, wv)
    it = fvv.Interpolator(blob(), 64, 64, precision=fvv.FVV_BF16, max_views=1)
    if kind == "conv":
        Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    else:
        Ho, Wo = 2 * H, 2 * W
    xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
    f32 = name not in BF16_OUT
    out = torch.full((n, Ho, Wo, co), -7.0, dtype=torch.float32 if f32 else torch.bfloat16, device="cuda")

    fvv.fvv_interp_inject_stall(it.h, STALL_CYCLES)
    fvv.fvv_interp_layer(it.h, li, xd, cs, 0, n, H, W, out, co, 0, f32)
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_interp_status(it.h)
    assert e.value.code == fvv.FVV_ETIMEOUT, e.value
    assert "code 6" in str(e.value), e.value
    assert (out.float().cpu().numpy() == -7).all(), "the stalled kernel wrote output"
    fvv.fvv_interp_status(it.h)                  # reading the status cleared the word

    fvv.fvv_interp_layer(it.h, li, xd, cs, 0, n, H, W, out, co, 0, f32)
    fvv.fvv_interp_status(it.h)
    got = out.float().cpu().numpy()
    for i in range(n):
        xi = x[i, ..., :ci]
        if kind == "conv":
            ref = oracle.conv3x3(xi, wq, bv, stride=stride, relu=relu)
        else:
            ref = oracle.conv_transpose4x4(xi, wq, bv, relu=relu)
        scale = max(1.0, float(np.abs(ref).max()))
        # (bf16 output: plus its rounding, 2^-8 relative at most)
        err = float((np.abs(got[i] - ref) - (0 if f32 else 2.0 ** -8) * np.abs(ref)).max())
        assert err <= 1e-4 * scale, (name, i, err, scale)
    it.close()


def test_inject_stall_rejects_bad_limits(torch_cuda):
    it = fvv.Interpolator(blob(), 64, 64, precision=fvv.FVV_BF16, max_views=1)
    for bad in (0, 999, 1 << 40):
        with pytest.raises(fvv.FvvError) as e:
            fvv.fvv_interp_inject_stall(it.h, bad)
        assert e.value.code == fvv.FVV_EINVAL
    it.close()
