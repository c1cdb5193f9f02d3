"""GPU parity of the halo path of the tensor-core convolutions.

3x3 stride-1 layers (and the all-phase transposed convs) with 128-byte operand
rows run, on grids at least 96 pixels wide, on tiles of one 128-pixel row whose
A operand is ONE box of 130 pixels per (row tap, channel block): the three
column taps read it 0, 1, 2 rows in.  Checks:

* each such layer (128-, 64- and 32-byte operand rows) alone on wide ragged grids (last tile partly outside the
  grid, zero padding on both sides) against the oracle's conv of the same
  bf16-rounded input and weights, the bar of the per-layer tests;
* the 256-channel layers on an odd tile count (one CTA per SM, each loading its
  own weight slices; a persistent CTA's last tile may be its only one);
* the stride-2 convs with 16/32-channel input pixels (one box of 129 pixel pairs per
  row tap, resident weights) on ragged grids against the oracle;
* the whole BF16 forward with the halo tiles equals, bit for bit, the same
  forward with every layer forced onto plain 1 x 128 tiles: both accumulate
  the K loop in the order (row tap, channel block, column tap), or (channel block,
  tap) for the per-phase transposed convs (the VIB t1 convs, whose column taps are
  folded into N and summed after the K loop, run on plain tiles in both);
* the forward with t1's folded column taps matches the one with t1 on plain tiles to
  FP32 rounding of that sum (stage flows, Eq. 2, and the views); so does the forward
  with RefineNet's output conv in its dedicated kernel (column taps folded into N,
  two rows of a 120-pixel strip per tile) against ref.out on plain tiles.

The transposed convs with C_out <= 32 (VIB t1, RefineNet d2, d3) run as one 3x3 conv
over all four output phases (N = 4 C_out); d2's phases are stored by TMA through the
pixel-pair map, one phase per staged chunk.  VIB t1 folds its three column taps into N
(N = 3 x 20 -> 64) on grids at least 256 wide: rows of 120 output pixels, four 32-pixel
boxes per (row tap, channel block); the layer tests run it on a grid 370 (= 3 x 120 + 10)
wide, and vib2.t1 on 131 keeps the per-row-tap boxes.
"""
import json

import numpy as np
import pytest

import oracle
import paper_2112_10603_b300 as fvv
from synth import weights
from tests.gpu_common import blob, pair

pytestmark = pytest.mark.gpu

# 128-byte rows (C_in >= 64), the narrow 32- / 64-byte rows (C_in = 16, 32; ref.out: an
# N = 16 tile with 3 real columns) and the all-phase transposed convs (t1, d3, and d2
# with TMA-stored phases)
HALO_LAYERS = ["vib2.m0", "vib0.m5", "vib2.t1", "ctx.c7", "ref.e1b", "ref.e3b", "ref.d3", "ctx.c1", "ctx.c3",
               "ref.e0b", "ref.d2", "ref.out", "vib1.t1"]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    return torch


def _bf16_round(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


@pytest.mark.parametrize("name", HALO_LAYERS)
def test_halo_layer_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    names = [m[0] for m in weights.manifest()]
    li = names.index(name)
    _, kind, ci, co, stride, relu = weights.manifest()[li]
    assert stride == 1 or kind == "convT"
    rng = np.random.default_rng(300 + li)
    # grid widths 260 = 2 x 128 + 4 (conv) and 131 = 128 + 3 (transposed conv input);
    # vib1.t1: 370 = 3 x 120 + 10 (four tiles of the folded column taps, grids >= 256)
    H, W = ((3, 370) if name == "vib1.t1" else (3, 131)) if kind == "convT" else (3, 260)
    # one image of vib2.m0: 3 x 3 = 9 tiles, an odd tile count for a 256-channel layer
    n = 1 if name == "vib2.m0" else 2
    cs = ci + (64 if li % 2 else 0)        # a wider pixel stride and a channel offset
    coff = 64 if li % 2 else 0
    x = np.zeros((n, H, W, cs), np.float32)
    x[..., coff:coff + ci] = rng.standard_normal((n, H, W, ci)) * 0.5
    x = _bf16_round(torch, x)
    wv, bv = weights.layer_views(blob())[name]
    wq = _bf16_round(torch, wv)
    it = fvv.Interpolator(blob(), 64, 64, precision=fvv.FVV_BF16, max_views=1)
    Ho, Wo = (2 * H, 2 * W) if kind == "convT" else (H, W)
    xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
    out = torch.full((n, Ho, Wo, co + 3), -7.0, dtype=torch.float32, device="cuda")
    fvv.fvv_interp_layer(it.h, li, xd, cs, coff, n, H, W, out, co + 3, 2, True)
    fvv.fvv_interp_status(it.h)
    got = out.cpu().numpy()
    assert (got[..., :2] == -7).all() and (got[..., 2 + co:] == -7).all(), "wrote outside its channel slot"
    for i in range(n):
        xi = x[i, ..., coff:coff + ci]
        if kind == "conv":
            ref = oracle.conv3x3(xi, wq, bv, stride=1, relu=relu)
        else:
            ref = oracle.conv_transpose4x4(xi, wq, bv, relu=relu)
        scale = max(1.0, float(np.abs(ref).max()))
        err = np.abs(got[i, ..., 2:2 + co] - ref).max()
        assert err <= 1e-4 * scale, (name, i, err, scale)


@pytest.mark.parametrize("name", ["ref.d2", "vib2.t0"])
def test_transposed_conv_tma_store_bf16(torch_cuda, name):
    """BF16 outputs of the transposed convs written through the pixel-pair TMA-store map:
    RefineNet d2 (all four phases in one tile, one staged chunk per phase) and VIB t0
    (one phase per tile), into a channel slot of a wider tensor."""
    torch = torch_cuda
    names = [m[0] for m in weights.manifest()]
    li = names.index(name)
    _, kind, ci, co, _, relu = weights.manifest()[li]
    rng = np.random.default_rng(700 + li)
    H, W, n = 3, 131, 2
    x = _bf16_round(torch, rng.standard_normal((n, H, W, ci)) * 0.5)
    wv, bv = weights.layer_views(blob())[name]
    wq = _bf16_round(torch, wv)
    it = fvv.Interpolator(blob(), 64, 64, precision=fvv.FVV_BF16, max_views=1)
    ocs, ooff = co + 32, 16
    xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
    out = torch.full((n, 2 * H, 2 * W, ocs), -7.0, dtype=torch.bfloat16, device="cuda")
    fvv.fvv_interp_layer(it.h, li, xd, ci, 0, n, H, W, out, ocs, ooff, False)
    fvv.fvv_interp_status(it.h)
    got = out.float().cpu().numpy()
    assert (got[..., :ooff] == -7).all() and (got[..., ooff + co:] == -7).all(), "wrote outside its channel slot"
    for i in range(n):
        ref = oracle.conv_transpose4x4(x[i], wq, bv, relu=relu)
        scale = max(1.0, float(np.abs(ref).max()))
        err = np.abs(got[i, ..., ooff:ooff + co] - ref) - np.abs(ref) * 2.0 ** -8
        assert err.max() <= 1e-4 * scale, (name, i, float(err.max()), scale)


# stride-2 convs whose input pixel is one 16- or 32-channel block: one box of 129 pixel
# pairs per row tap feeds the three column taps, weights resident in shared memory
# (vib2.c0, 32 -> 128, keeps the per-tap tiles: the same wide ragged grid on that path)
S2H_LAYERS = ["vib0.c0", "ref.e0a", "ctx.c2", "ctx.c4", "vib2.c0"]


@pytest.mark.parametrize("name", S2H_LAYERS)
def test_stride2_pair_halo_layer_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    names = [m[0] for m in weights.manifest()]
    li = names.index(name)
    _, kind, ci, co, stride, relu = weights.manifest()[li]
    assert stride == 2 and kind == "conv"
    rng = np.random.default_rng(500 + li)
    # output grid 3 x 132 = one full and one ragged 128-pixel tile per row; the input
    # pixel stride is the padded channel block (16 or 32), its pad channels zero
    H, W, n = 6, 264, 2
    cs = 16 if ci <= 16 else 32
    x = np.zeros((n, H, W, cs), np.float32)
    x[..., :ci] = rng.standard_normal((n, H, W, ci)) * 0.5
    x = _bf16_round(torch, x)
    wv, bv = weights.layer_views(blob())[name]
    wq = _bf16_round(torch, wv)
    it = fvv.Interpolator(blob(), 64, 64, precision=fvv.FVV_BF16, max_views=1)
    Ho, Wo = H // 2, W // 2
    xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
    out = torch.full((n, Ho, Wo, co + 3), -7.0, dtype=torch.float32, device="cuda")
    fvv.fvv_interp_layer(it.h, li, xd, cs, 0, n, H, W, out, co + 3, 2, True)
    fvv.fvv_interp_status(it.h)
    got = out.cpu().numpy()
    assert (got[..., :2] == -7).all() and (got[..., 2 + co:] == -7).all(), "wrote outside its channel slot"
    for i in range(n):
        ref = oracle.conv3x3(x[i, ..., :ci], wq, bv, stride=2, relu=relu)
        scale = max(1.0, float(np.abs(ref).max()))
        err = np.abs(got[i, ..., 2:2 + co] - ref).max()
        assert err <= 1e-4 * scale, (name, i, err, scale)


def test_halo_network_bitwise_plain_tiles(torch_cuda, tmp_path):
    torch = torch_cuda
    # 64 x 512: VIB2's 256-channel convs, vib2.t1, ref.e1b and ref.d3 take halo tiles;
    # RefineNet e0a and ContextNet c2 take stride-2 pair-halo tiles
    H, W = 64, 512
    left, right = pair(21, H, W, 10.0)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ts = [0.3, 0.8]
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=2)
    key = f"{H}x{W} n2 p{fvv.FVV_BF16}"
    # t1 (folded column taps) on plain tiles, every other layer on its default tiles
    t1_plain = tmp_path / "t1.json"
    # (and the output conv and d3: their dedicated kernels fold the column taps too)
    t1_plain.write_text(json.dumps({key: {**{f"vib{s}.t1": 7 for s in range(3)}, "ref.out": 7, "ref.d3": 7}}))
    it.autotune(2, str(t1_plain))
    halo = it.run(L, R, ts).cpu().numpy()
    # force every layer onto plain tiles 128 pixels wide through a tile cache entry
    cache = tmp_path / "plain.json"
    cache.write_text(json.dumps({key: {m[0]: 7 for m in weights.manifest()}}))
    it.autotune(2, str(cache))
    plain = it.run(L, R, ts).cpu().numpy()
    fvv.fvv_interp_status(it.h)
    np.testing.assert_array_equal(halo, plain)


def test_folded_t1_network_matches_plain_t1(torch_cuda, tmp_path):
    """VIB t1 with its column taps folded into N against t1 on plain tiles, the rest of
    the network unchanged: the two differ only in the FP32 order of the three column
    taps' sums, so the stage flows (Eq. 2 fused into t1) agree to far below a pixel and
    the views to BF16 noise."""
    torch = torch_cuda
    H, W = 64, 512
    left, right = pair(23, H, W, 10.0)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ts = [0.4, 0.7]
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=2)
    folded = it.run(L, R, ts).cpu().numpy()
    flows = [it.peek(f"vib{s}").copy() for s in range(3)]
    cache = tmp_path / "t1.json"
    cache.write_text(json.dumps({f"{H}x{W} n2 p{fvv.FVV_BF16}": {f"vib{s}.t1": 7 for s in range(3)}}))
    it.autotune(2, str(cache))
    plain = it.run(L, R, ts).cpu().numpy()
    fvv.fvv_interp_status(it.h)
    for s in range(3):
        d = np.abs(it.peek(f"vib{s}") - flows[s])
        assert d.max() < 0.05, (s, float(d.max()))
    d = np.abs(folded - plain)
    assert d.max() < 0.05 and d.mean() < 1e-3, (float(d.max()), float(d.mean()))


@pytest.mark.parametrize("H,W,nv", [(71, 399, 2), (64, 512, 3)])
def test_folded_output_conv_matches_plain(torch_cuda, tmp_path, H, W, nv):
    """RefineNet's output conv and d3 in their dedicated kernels (column taps folded into
    N, the three taps summed across TMEM lanes, tiles walking down 120-pixel strips)
    against the generic tensor-core convs on plain tiles (a tile width forced for ref.out
    and ref.d3 in the tile cache), the rest of the network unchanged: the two differ only
    in the FP32 order of the taps' sums (and d3's bf16 rounding of them), so every
    earlier intermediate is the same and the views agree to far below BF16 noise.  Odd
    crop height (the last row pair half outside), odd crop width (scalar stores), ragged
    last strips."""
    torch = torch_cuda
    left, right = pair(29, H, W, 8.0)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ts = [0.25, 0.5, 0.75][:nv]
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=nv)
    folded = it.run(L, R, ts).cpu().numpy()
    blend = it.peek("blend").copy()
    cache = tmp_path / "out.json"
    cache.write_text(json.dumps({f"{H}x{W} n{nv} p{fvv.FVV_BF16}": {"ref.out": 7, "ref.d3": 7}}))
    it.autotune(nv, str(cache))
    plain = it.run(L, R, ts).cpu().numpy()
    fvv.fvv_interp_status(it.h)
    np.testing.assert_array_equal(it.peek("blend"), blend)
    assert folded.shape == (nv, H, W, 3) and np.isfinite(folded).all()
    d = np.abs(folded - plain)
    assert d.max() <= 2e-3 and d.mean() <= 2e-5, (float(d.max()), float(d.mean()))


@pytest.mark.parametrize("H,W,n", [(3, 131, 2), (5, 250, 1)])
def test_folded_d3_layer_matches_oracle(torch_cuda, H, W, n):
    """ref.d3 (all-phase transposed conv 64 -> 16, ReLU) in its dedicated kernel (column
    taps folded into N = 192): bf16 input in the network's 96-channel pixel stride, bf16
    output of pitch 16, against the oracle's transposed conv of the same bf16-rounded
    operands (the per-layer bar plus the output's bf16 rounding); ragged strips (131 =
    120 + 11, 250 = 2 x 120 + 10) and rows walked down each strip."""
    torch = torch_cuda
    names = [m[0] for m in weights.manifest()]
    li = names.index("ref.d3")
    _, kind, ci, co, _, relu = weights.manifest()[li]
    assert (kind, ci, co, relu) == ("convT", 64, 16, True)
    rng = np.random.default_rng(900 + H)
    x = np.zeros((n, H, W, 96), np.float32)
    x[..., :ci] = rng.standard_normal((n, H, W, ci)) * 0.5
    x = _bf16_round(torch, x)
    wv, bv = weights.layer_views(blob())["ref.d3"]
    wq = _bf16_round(torch, wv)
    it = fvv.Interpolator(blob(), 64, 64, precision=fvv.FVV_BF16, max_views=1)
    xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
    out = torch.full((n, 2 * H, 2 * W, co), -7.0, dtype=torch.bfloat16, device="cuda")
    fvv.fvv_interp_layer(it.h, li, xd, 96, 0, n, H, W, out, co, 0, False)
    fvv.fvv_interp_status(it.h)
    got = out.float().cpu().numpy()
    for i in range(n):
        ref = oracle.conv_transpose4x4(x[i, ..., :ci], wq, bv, relu=True)
        scale = max(1.0, float(np.abs(ref).max()))
        err = np.abs(got[i] - ref) - np.abs(ref) * 2.0 ** -8
        assert err.max() <= 1e-4 * scale, (i, float(err.max()), scale)


@pytest.mark.parametrize("H,W,nv", [(72, 400, 3), (200, 136, 2)])
def test_stage_input_in_c0_loader_bitwise(torch_cuda, tmp_path, H, W, nv):
    """VIB1/VIB2 c0 with the stage input computed by its loader warps (never stored)
    against the stage-input kernel followed by the per-tap c0 (a tile width forced for
    the two c0 layers in the tile cache turns the fusion off): the same bits, on ragged
    column strips (400 wide: VIB2 c0 outputs 200 = 126 + 74 per row), several views and
    tile ranges that cross strips and views."""
    torch = torch_cuda
    left, right = pair(31, H, W, 9.0)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ts = [0.2, 0.5, 0.9][:nv]
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=nv)
    fused = it.run(L, R, ts).cpu().numpy()
    flows = [it.peek(f"vib{s}").copy() for s in range(3)]
    cache = tmp_path / "c0.json"
    cache.write_text(json.dumps({f"{H}x{W} n{nv} p{fvv.FVV_BF16}": {"vib1.c0": 7, "vib2.c0": 7}}))
    it.autotune(nv, str(cache))
    apart = it.run(L, R, ts).cpu().numpy()
    fvv.fvv_interp_status(it.h)
    for s in range(3):
        np.testing.assert_array_equal(it.peek(f"vib{s}"), flows[s])
    np.testing.assert_array_equal(apart, fused)
