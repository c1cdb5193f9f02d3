"""Pins of the oracle's building blocks against library routines, closed forms
and invariants (CPU only).

* conv / convT / box / upsample / warp against float64 torch.nn.functional
  (conv2d, conv_transpose2d, avg_pool2d, interpolate, grid_sample): special
  cases that reduce to a library routine;
* warp: zero flow is the identity, a constant image stays constant, an integer
  flow in circular mode is a pure cyclic shift (exact);
* blend (Eq. 1): a mask of 1 / 0 returns exactly one input;
* hand-computed closed forms on 1-pixel-wide cases.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

import oracle

RTOL = 1e-12


def _nchw(x):
    return torch.from_numpy(np.ascontiguousarray(x)).permute(2, 0, 1)[None].double()


def _hwc(t):
    return t[0].permute(1, 2, 0).numpy()


def _rand(rng, *shape):
    return rng.standard_normal(shape)


@pytest.mark.parametrize("H,W,Ci,Co,stride,circ", [
    (5, 7, 3, 4, 1, False), (5, 7, 3, 4, 2, False), (6, 8, 5, 3, 2, True),
    (4, 4, 2, 6, 1, True), (9, 3, 1, 1, 2, False), (1, 1, 4, 2, 1, False),
])
def test_conv3x3_matches_torch(H, W, Ci, Co, stride, circ):
    rng = np.random.default_rng(H * 100 + W)
    x = _rand(rng, H, W, Ci)
    w = _rand(rng, Co, Ci, 3, 3).astype(np.float32)
    b = _rand(rng, Co).astype(np.float32)
    got = oracle.conv3x3(x, w, b, stride=stride, circ=circ)
    xt = _nchw(x)
    wt, bt = torch.from_numpy(w).double(), torch.from_numpy(b).double()
    if circ:
        ref = Fn.conv2d(Fn.pad(xt, (1, 1, 1, 1), mode="circular"), wt, bt, stride=stride)
    else:
        ref = Fn.conv2d(xt, wt, bt, stride=stride, padding=1)
    np.testing.assert_allclose(got, _hwc(ref), rtol=RTOL, atol=1e-12)
    got_r = oracle.conv3x3(x, w, b, stride=stride, circ=circ, relu=True)
    np.testing.assert_allclose(got_r, np.maximum(_hwc(ref), 0), rtol=RTOL, atol=1e-12)


@pytest.mark.parametrize("H,W,Ci,Co,circ", [
    (3, 5, 2, 3, False), (4, 4, 3, 5, False), (1, 1, 2, 2, False), (3, 4, 2, 3, True), (2, 5, 1, 4, True),
])
def test_convT_matches_torch(H, W, Ci, Co, circ):
    rng = np.random.default_rng(7 * H + W)
    x = _rand(rng, H, W, Ci)
    w = _rand(rng, Ci, Co, 4, 4).astype(np.float32)
    b = _rand(rng, Co).astype(np.float32)
    got = oracle.conv_transpose4x4(x, w, b, circ=circ)
    xt = _nchw(x)
    wt, bt = torch.from_numpy(w).double(), torch.from_numpy(b).double()
    if circ:
        # circular transposed conv = full transposed conv of the circularly padded
        # input, cropped so that output o maps to full index o + 3
        full = Fn.conv_transpose2d(Fn.pad(xt, (1, 1, 1, 1), mode="circular"), wt, bt, stride=2)
        ref = full[..., 3:3 + 2 * H, 3:3 + 2 * W]
    else:
        ref = Fn.conv_transpose2d(xt, wt, bt, stride=2, padding=1)
    assert ref.shape[-2:] == (2 * H, 2 * W)
    np.testing.assert_allclose(got, _hwc(ref), rtol=RTOL, atol=1e-12)


def test_convT_single_pixel_closed_form():
    # one input pixel, one channel: output (2x2) = b + x * w[1:3, 1:3] (taps ky, kx in {1, 2})
    w = np.arange(16, dtype=np.float32).reshape(1, 1, 4, 4)
    b = np.array([0.5], np.float32)
    got = oracle.conv_transpose4x4(np.full((1, 1, 1), 2.0), w, b)[..., 0]
    np.testing.assert_array_equal(got, 0.5 + 2.0 * w[0, 0, 1:3, 1:3])


def test_conv_center_tap_closed_form():
    # only the centre tap set: conv is a per-pixel linear map of channels
    rng = np.random.default_rng(3)
    x = _rand(rng, 4, 6, 3)
    w = np.zeros((2, 3, 3, 3), np.float32)
    w[:, :, 1, 1] = rng.standard_normal((2, 3)).astype(np.float32)
    b = np.array([0.25, -1.0], np.float32)
    got = oracle.conv3x3(x, w, b)
    np.testing.assert_allclose(got, x @ w[:, :, 1, 1].T.astype(np.float64) + b, rtol=1e-14, atol=1e-14)
    got2 = oracle.conv3x3(x, w, b, stride=2)
    np.testing.assert_allclose(got2, (x @ w[:, :, 1, 1].T.astype(np.float64) + b)[::2, ::2], rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("f", [2, 4])
def test_box_down_matches_avg_pool(f):
    rng = np.random.default_rng(f)
    x = _rand(rng, 8, 12, 5)
    got = oracle.box_down(x, f)
    ref = _hwc(Fn.avg_pool2d(_nchw(x), f))
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-15)


def test_upsample_matches_interpolate():
    rng = np.random.default_rng(11)
    x = _rand(rng, 5, 7, 4)
    got = oracle.upsample2x(x)
    ref = _hwc(Fn.interpolate(_nchw(x), scale_factor=2, mode="bilinear", align_corners=False))
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=1e-13)


def test_upsample_circular_matches_padded_interpolate():
    rng = np.random.default_rng(12)
    H, W = 4, 6
    x = _rand(rng, H, W, 2)
    got = oracle.upsample2x(x, circ=True)
    # wrap-padding by one coarse pixel and cropping two fine pixels gives the wrapped taps
    big = Fn.interpolate(Fn.pad(_nchw(x), (1, 1, 1, 1), mode="circular"), scale_factor=2,
                         mode="bilinear", align_corners=False)
    ref = _hwc(big[..., 2:2 + 2 * H, 2:2 + 2 * W])
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=1e-13)


def test_upsample_weights_closed_form():
    # 1-D ramp: interior fine pixels are 0.25 / 0.75 mixes of their coarse neighbours
    x = np.arange(6, dtype=np.float64).reshape(1, 6, 1)
    got = oracle.upsample2x(x)[0, :, 0]
    exp_ = [0.0, 0.25, 0.75, 1.25, 1.75, 2.25, 2.75, 3.25, 3.75, 4.25, 4.75, 5.0]
    np.testing.assert_allclose(got, exp_, rtol=0, atol=1e-15)


def _grid_sample_border(img, flow):
    H, W, _ = img.shape
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    gx = (xs + flow[..., 0] + 0.5) / W * 2 - 1
    gy = (ys + flow[..., 1] + 0.5) / H * 2 - 1
    grid = torch.from_numpy(np.stack([gx, gy], -1))[None]
    return _hwc(Fn.grid_sample(_nchw(img), grid, mode="bilinear", padding_mode="border",
                               align_corners=False))


@pytest.mark.parametrize("scale", [0.7, 3.0, 40.0])
def test_warp_matches_grid_sample_border(scale):
    rng = np.random.default_rng(int(scale * 10))
    img = _rand(rng, 9, 13, 3)
    flow = _rand(rng, 9, 13, 2) * scale
    got = oracle.warp(img, flow)
    np.testing.assert_allclose(got, _grid_sample_border(img, flow), rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("circ", [False, True])
def test_warp_zero_flow_is_identity(circ):
    rng = np.random.default_rng(5)
    img = _rand(rng, 6, 9, 4)
    np.testing.assert_array_equal(oracle.warp(img, np.zeros((6, 9, 2)), circ=circ), img)


@pytest.mark.parametrize("circ", [False, True])
def test_warp_constant_image_stays_constant(circ):
    rng = np.random.default_rng(6)
    img = np.full((7, 5, 3), 0.37)
    flow = _rand(rng, 7, 5, 2) * 4
    np.testing.assert_allclose(oracle.warp(img, flow, circ=circ), img, rtol=0, atol=1e-15)


def test_warp_integer_flow_circular_is_roll():
    rng = np.random.default_rng(8)
    img = _rand(rng, 8, 10, 2)
    flow = np.zeros((8, 10, 2))
    flow[..., 0], flow[..., 1] = 3, -2
    # out(y, x) = img(y - 2, x + 3)
    np.testing.assert_array_equal(oracle.warp(img, flow, circ=True),
                                  np.roll(img, shift=(2, -3), axis=(0, 1)))


def test_warp_half_pixel_closed_form():
    img = np.arange(4, dtype=np.float64).reshape(1, 4, 1)
    flow = np.zeros((1, 4, 2))
    flow[..., 0] = 0.5
    # samples at x + 0.5 on a ramp; the last pixel clamps to the border value 3
    np.testing.assert_allclose(oracle.warp(img, flow)[0, :, 0], [0.5, 1.5, 2.5, 3.0], atol=1e-15)


def test_blend_mask_one_and_zero():
    rng = np.random.default_rng(9)
    a, b = _rand(rng, 5, 6, 3), _rand(rng, 5, 6, 3)
    np.testing.assert_array_equal(oracle.blend(a, b, np.ones((5, 6))), a)
    np.testing.assert_array_equal(oracle.blend(a, b, np.zeros((5, 6))), b)
    np.testing.assert_allclose(oracle.blend(a, b, np.full((5, 6), 0.5)), 0.5 * (a + b), atol=1e-15)
