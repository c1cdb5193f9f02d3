"""FP8 (E4M3) path: every VIBlock conv with 128 or 256 input channels (c1, the six
256-channel convs m0-m5, the transposed t0 and t1) with per-output-channel weight scales
and calibrated per-tensor activation scales, FP32 accumulation.

Kernel level: an FP8 layer on E4M3 input codes equals the oracle's conv of the
dequantised operands (codes x scales): a product of two E4M3 values is exact in
FP32, so only the summation order differs (|err| <= 1e-4 x output scale).
Network level: PSNR against the FP64 oracle is reported and held to a floor."""
import numpy as np
import pytest

import oracle
import paper_2112_10603_b300 as fvv
from synth import scene, weights
from tests.gpu_common import blob, oracle_view, pair, psnr

pytestmark = pytest.mark.gpu
# 256x256, seed 1: 34.6-34.8 dB over three scenes and five calibration sets.  The E4M3
# rounding of weights and activations (relative step 2^-3) leaves 10-13% RMS relative
# error in the stage flows at every size; the 256x256 scenes have about 7x the per-pixel
# image gradient of the 1080p ones, so the same flow error costs ~6 dB more there
# (1080p: 40.7 dB, held to the 38 dB target below).
PSNR_FP8_FLOOR = 34.0
# Circular padding, same scenes: 32.8-32.9 dB.  The stage flows carry the same relative
# error (0.09-0.13); the loss is at the wrapped seams, where the non-periodic scene's
# opposite edges meet (mean error in the 4 border pixels 0.038-0.041 against 0.010-0.012
# with zero padding, interior 0.014 against 0.012; BF16 loses ~1 dB there too).
PSNR_FP8_CIRC_FLOOR = 32.0
FLOW_REL_ERR_MAX = 0.14   # RMS flow error / RMS flow, each stage s of Eq. 2


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    return torch


def _calib_frames(torch, H, W, seeds=(100, 101)):
    fr = []
    for s in seeds:
        l, r = scene.stereo_pair(s, H, W, 6.0 if W < 400 else 64.0)
        fr += [l, r]
    return torch.from_numpy(np.stack(fr)).cuda()


def _e4m3(torch, x):
    """E4M3 codes (uint8) and their values, round to nearest even."""
    t = torch.from_numpy(np.clip(x, -448, 448).astype(np.float32)).to(torch.float8_e4m3fn)
    return t.view(torch.uint8).numpy(), t.to(torch.float32).numpy()


def test_fp8_requires_calibration(torch_cuda):
    torch = torch_cuda
    it = fvv.Interpolator(blob(), 64, 96, precision=fvv.FVV_FP8, max_views=1)
    x = torch.zeros(64, 96, 3, device="cuda")
    with pytest.raises(fvv.FvvError) as e:
        it.run(x, x, [0.5])
    assert e.value.code == fvv.FVV_EINVAL


# (19, 42): 8 x 16 tiles; (3, 200): one-row halo tiles (130-pixel A boxes), ragged tail
@pytest.mark.parametrize("h,ww", [(19, 42), (3, 200)])
@pytest.mark.parametrize("name", ["vib1.m0", "vib2.m3", "vib0.m5"])
def test_fp8_layer_matches_dequantised_oracle(torch_cuda, name, h, ww):
    torch = torch_cuda
    H, W = 64, 96
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_FP8, max_views=3)
    fvv.fvv_calibrate_fp8(it.h, _calib_frames(torch, H, W), 2)
    li = [m[0] for m in weights.manifest()].index(name)
    s_a, s_w = fvv.fvv_interp_fp8_scales(it.h, li, 256)
    assert s_a > 0 and (s_w > 0).all()
    w, b = weights.layer_views(blob())[name]
    wq_codes, wq = _e4m3(torch, w / s_w[:, None, None, None])
    rng = np.random.default_rng(li)
    n = 2
    x = np.maximum(rng.standard_normal((n, h, ww, 256)), 0) * (100 * s_a)
    xq_codes, xq = _e4m3(torch, x / s_a)
    xd = torch.from_numpy(np.ascontiguousarray(xq_codes)).cuda()
    out = torch.zeros((n, h, ww, 256), device="cuda")
    fvv.fvv_interp_layer(it.h, li, xd, 256, 0, n, h, ww, out, 256, 0, True)
    fvv.fvv_interp_status(it.h)
    got = out.cpu().numpy()
    for i in range(n):
        ref = oracle.conv3x3(xq[i].astype(np.float64) * s_a, wq * s_w[:, None, None, None], b, relu=True)
        scale = max(1.0, float(np.abs(ref).max()))
        assert np.abs(got[i] - ref).max() <= 1e-4 * scale


@pytest.mark.parametrize("name", ["vib2.c1", "vib0.c1", "vib1.t0", "vib2.t0", "vib2.t1", "vib0.t1"])
def test_fp8_strided_and_transposed_layers(torch_cuda, name):
    """The stride-2 c1 (128 -> 256), the transposed t0 (256 -> 128) and the all-phase
    transposed t1 (128 -> 5) on E4M3 codes equal the oracle's conv of the dequantised
    operands, ragged tiles included."""
    torch = torch_cuda
    H, W = 64, 96
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_FP8, max_views=3)
    fvv.fvv_calibrate_fp8(it.h, _calib_frames(torch, H, W), 2)
    li = [m[0] for m in weights.manifest()].index(name)
    _, kind, ci, co, stride, relu = weights.manifest()[li]
    s_a, s_w = fvv.fvv_interp_fp8_scales(it.h, li, co)
    assert s_a > 0 and (s_w > 0).all()
    w, b = weights.layer_views(blob())[name]
    # per output channel: conv weights are [C_out][C_in][3][3], transposed [C_in][C_out][4][4]
    sw = s_w[:, None, None, None] if kind == "conv" else s_w[None, :, None, None]
    wq_codes, wq = _e4m3(torch, w / sw)
    rng = np.random.default_rng(li)
    # vib2.t1 also on a wider grid, 370 = 2 x 128 + 114
    n, h, ww = 2, (6 if kind == "conv" else 3), (260 if kind == "conv" else (370 if name == "vib2.t1" else 131))
    x = np.maximum(rng.standard_normal((n, h, ww, ci)), 0) * (100 * s_a)
    xq_codes, xq = _e4m3(torch, x / s_a)
    xd = torch.from_numpy(np.ascontiguousarray(xq_codes)).cuda()
    Ho, Wo = (h // 2, ww // 2) if kind == "conv" else (2 * h, 2 * ww)
    out = torch.zeros((n, Ho, Wo, co), device="cuda")
    fvv.fvv_interp_layer(it.h, li, xd, ci, 0, n, h, ww, out, co, 0, True)
    fvv.fvv_interp_status(it.h)
    got = out.cpu().numpy()
    for i in range(n):
        xi = xq[i].astype(np.float64) * s_a
        if kind == "conv":
            ref = oracle.conv3x3(xi, wq * sw, b, stride=2, relu=relu)
        else:
            ref = oracle.conv_transpose4x4(xi, wq * sw, b, relu=relu)
        scale = max(1.0, float(np.abs(ref).max()))
        assert np.abs(got[i] - ref).max() <= 1e-4 * scale, (name, i)


@pytest.mark.parametrize("H,W,seed,disp", [(256, 256, 1, 12.0)])
def test_fp8_network_psnr(torch_cuda, H, W, seed, disp):
    torch = torch_cuda
    left, right = pair(seed, H, W, disp)
    ref, d = oracle_view(seed, H, W, disp, 0.5)
    it8 = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_FP8, max_views=3)
    fvv.fvv_calibrate_fp8(it8.h, _calib_frames(torch, H, W), 2)
    it16 = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=1)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    o8 = it8.run(L, R, [0.5]).cpu().numpy()[0]
    o16 = it16.run(L, R, [0.5]).cpu().numpy()[0]
    p8, p816 = psnr(o8, ref), psnr(o8, o16)
    print(f"FP8 {H}x{W}: PSNR {p8:.2f} dB vs FP64, {p816:.2f} dB vs BF16, max err {np.abs(o8 - ref).max():.4f}")
    assert np.isfinite(o8).all() and o8.min() >= 0 and o8.max() <= 1
    assert p8 >= PSNR_FP8_FLOOR, p8
    for s in range(3):
        g, r = it8.peek(f"vib{s}")[..., :4], d[f"vib{s}"][..., :4]
        rel = np.sqrt(((g - r) ** 2).mean() / (r ** 2).mean())
        print(f"  stage {s}: flow RMS relative error {rel:.3f}")
        assert rel <= FLOW_REL_ERR_MAX, (s, rel)


def test_fp8_1080p_fifteen_views(torch_cuda):
    """1920x1080, 15 views at t = k/16, calibration on 8 held-out scenes (seeds
    100-107): the midpoint view reaches 38 dB against the FP64 oracle with its stage
    flows within the same relative error as at 256x256, every view is finite and in
    [0, 1], and each view equals the same view computed alone."""
    torch = torch_cuda
    H, W = 1080, 1920
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_FP8, max_views=15)
    fvv.fvv_calibrate_fp8(it.h, _calib_frames(torch, H, W, seeds=range(100, 108)), 8)
    left, right = pair(2, H, W, 64.0)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ts = [k / 16 for k in range(1, 16)]
    out = it.run(L, R, ts).cpu().numpy()
    fvv.fvv_interp_status(it.h)
    assert np.isfinite(out).all() and out.min() >= 0 and out.max() <= 1
    ref, d = oracle_view(2, H, W, 64.0, 0.5)
    p = psnr(out[7], ref)
    print(f"FP8 1080p t=0.5 (15-view batch): PSNR {p:.2f} dB")
    assert p >= 38.0, p
    for s in range(3):
        g, r = it.peek(f"vib{s}", view=7)[..., :4], d[f"vib{s}"][..., :4]
        rel = np.sqrt(((g - r) ** 2).mean() / (r ** 2).mean())
        assert rel <= FLOW_REL_ERR_MAX, (s, rel)
    alone = it.run(L, R, [ts[3]]).cpu().numpy()
    np.testing.assert_array_equal(alone[0], out[3])


def test_fp8_circular_mode_and_shift_equivariance(torch_cuda):
    """E4M3 layers with circular padding (the wrapped-border copies of every conv input
    feed the E4M3 kernels as they feed the BF16 ones; calibration runs in the same mode):
    the view against the circular FP64 oracle at this size's circular FP8 floor, the stage flows
    within the same relative error bound, and shifting both frames cyclically by multiples
    of 16 pixels shifts the view bit for bit (the scales are fixed by calibration, so every
    element's arithmetic is the same wherever it lies)."""
    torch = torch_cuda
    H, W, seed, disp = 256, 256, 1, 12.0
    left, right = pair(seed, H, W, disp)
    ref, d = oracle_view(seed, H, W, disp, 0.5, circ=True)
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_FP8, max_views=1, pad_mode=fvv.FVV_PAD_CIRCULAR)
    fvv.fvv_calibrate_fp8(it.h, _calib_frames(torch, H, W), 2)
    a = it.run(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), [0.5]).cpu().numpy()[0]
    p = psnr(a, ref)
    print(f"FP8 circular {H}x{W}: PSNR {p:.2f} dB vs FP64")
    assert np.isfinite(a).all() and a.min() >= 0 and a.max() <= 1
    assert p >= PSNR_FP8_CIRC_FLOOR, p
    for s in range(3):
        g, r = it.peek(f"vib{s}")[..., :4], d[f"vib{s}"][..., :4]
        rel = np.sqrt(((g - r) ** 2).mean() / (r ** 2).mean())
        assert rel <= FLOW_REL_ERR_MAX, (s, rel)
    shift = (32, -80)
    Ls = torch.from_numpy(np.ascontiguousarray(np.roll(left, shift, (0, 1)))).cuda()
    Rs = torch.from_numpy(np.ascontiguousarray(np.roll(right, shift, (0, 1)))).cuda()
    b = it.run(Ls, Rs, [0.5]).cpu().numpy()[0]
    fvv.fvv_interp_status(it.h)
    it.close()
    np.testing.assert_array_equal(np.roll(a, shift, (0, 1)), b)
