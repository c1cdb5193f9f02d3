"""Batched execution: CUDA-graph replay, the tile autotuner, the rig batch call.

* graph replay (opts.graphs = 1) equals direct launches bit for bit, also when the
  output buffer, the t values and the camera frames change between replays;
* autotuned tile rectangles change no output bit (every output element keeps the
  same K-loop order whatever the tile) and the JSON cache round-trips;
* a rig instant with uneven per-pair view counts (one batch) equals per-pair runs;
* every view of such a rig instant matches the FP64 oracle's view of its pair:
  FP32 path max |err| <= 1e-4, BF16 path PSNR >= 45 dB;
* ContextNet on its own stream beside the VIBlocks (the default) gives the same bits as
  the whole forward on one stream (profiling mode runs it so).
"""
import json

import numpy as np
import pytest

import oracle
import paper_2112_10603_b300 as fvv
from synth import scene
from tests.gpu_common import blob, pair, psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    return torch


@pytest.mark.parametrize("precision", [fvv.FVV_FP32, fvv.FVV_BF16])
def test_graph_replay_is_bitwise_direct(torch_cuda, precision):
    torch = torch_cuda
    H, W = 72, 100
    l1, r1 = pair(11, H, W, 6.0)
    l2, r2 = pair(12, H, W, 6.0)
    g = fvv.Interpolator(blob(), H, W, precision=precision, max_views=3, graphs=1)
    d = fvv.Interpolator(blob(), H, W, precision=precision, max_views=3, graphs=0)
    for (l, r, ts) in ((l1, r1, [0.2, 0.7, 0.5]), (l2, r2, [0.9, 0.1, 0.4]), (l1, r1, [0.3, 0.3, 0.6])):
        L, R = torch.from_numpy(l).cuda(), torch.from_numpy(r).cuda()
        a = g.run(L, R, ts).cpu().numpy()          # a fresh output buffer every call
        b = d.run(L, R, ts).cpu().numpy()
        np.testing.assert_array_equal(a, b)
    fvv.fvv_interp_status(g.h)


def test_autotune_keeps_bits_and_caches(torch_cuda, tmp_path):
    torch = torch_cuda
    H, W = 72, 100
    left, right = pair(13, H, W, 6.0)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ts = [0.25, 0.5, 0.75]
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=3)
    before = it.run(L, R, ts).cpu().numpy()
    cache = tmp_path / "tiles.json"
    it.autotune(3, str(cache))
    after = it.run(L, R, ts).cpu().numpy()
    np.testing.assert_array_equal(before, after)
    data = json.loads(cache.read_text())
    key = f"{H}x{W} n3 p{fvv.FVV_BF16}"
    assert key in data and data[key]["vib2.m0"] in (-1, 3, 4, 5, 6, 7, 8)   # -1 = default rectangle
    it2 = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=3)
    it2.autotune(3, str(cache))                  # loaded from the cache
    np.testing.assert_array_equal(it2.run(L, R, ts).cpu().numpy(), before)


def test_rig_instant_uneven_counts(torch_cuda):
    torch = torch_cuda
    H, W = 48, 80
    cams = [torch.from_numpy(c).cuda() for c in scene.rig(14, H, W, n_cams=5, max_disp=6.0)]
    rng = np.random.default_rng(14)
    counts = [3, 1, 4, 2]
    offs = np.concatenate([[0], np.cumsum(counts)])
    ts = np.concatenate([np.sort(rng.uniform(0, 1, c)) for c in counts]).astype(np.float32)
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=16, max_cams=5)
    out = it.run_batch(cams, [0, 1, 2, 3], offs, ts).cpu().numpy()
    one = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=4)
    for p in range(4):
        ref = one.run(cams[p], cams[p + 1], ts[offs[p]:offs[p + 1]]).cpu().numpy()
        np.testing.assert_array_equal(out[offs[p]:offs[p + 1]], ref)


def test_rig_1080p_batch_equals_per_pair_runs(torch_cuda):
    """The rig configuration's launch shape: 1920 x 1080 frames of a 4-camera arc, three
    pairs with uneven view counts in one batched call (BF16, graph replay) equal the
    per-pair calls bit for bit (every layer's per-pixel arithmetic is the same whatever
    the batch and its size bucket)."""
    torch = torch_cuda
    H, W = 1080, 1920
    cams = [torch.from_numpy(c).cuda() for c in scene.rig(4, H, W, n_cams=4, max_disp=64.0)]
    counts = [3, 1, 2]
    offs = np.concatenate([[0], np.cumsum(counts)])
    ts = np.array([0.2, 0.5, 0.9, 0.4, 0.1, 0.7], np.float32)
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=6, max_cams=4)
    out = it.run_batch(cams, [0, 1, 2], offs, ts).cpu().numpy()
    fvv.fvv_interp_status(it.h)
    it.close()
    one = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=3)
    for p in range(3):
        ref = one.run(cams[p], cams[p + 1], ts[offs[p]:offs[p + 1]]).cpu().numpy()
        np.testing.assert_array_equal(out[offs[p]:offs[p + 1]], ref)
    one.close()


def test_rig_instant_with_an_empty_pair(torch_cuda):
    """A rig instant in which one pair asks for no views (view_offsets repeats an entry):
    the other pairs' views equal per-pair runs bit for bit and the FP64 oracle's views
    within 1e-4 (FP32 path); a call with no views at all is refused (FVV_ESHAPE)."""
    torch = torch_cuda
    H, W = 40, 72
    frames = scene.rig(17, H, W, n_cams=5, max_disp=6.0)
    cams = [torch.from_numpy(c).cuda() for c in frames]
    counts = [2, 0, 1, 2]
    offs = np.concatenate([[0], np.cumsum(counts)])
    ts = np.array([0.3, 0.8, 0.5, 0.1, 0.9], np.float32)
    it = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_FP32, max_views=8, max_cams=5)
    out = it.run_batch(cams, [0, 1, 2, 3], offs, ts).cpu().numpy()
    one = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_FP32, max_views=4)
    for p in range(4):
        if counts[p] == 0:
            continue
        ref = one.run(cams[p], cams[p + 1], ts[offs[p]:offs[p + 1]]).cpu().numpy()
        np.testing.assert_array_equal(out[offs[p]:offs[p + 1]], ref)
        for v in range(offs[p], offs[p + 1]):
            o = oracle.vinet_forward(blob(), frames[p], frames[p + 1], float(ts[v]))
            assert float(np.abs(out[v] - o).max()) <= 1e-4, v
    dev_out = torch.empty((1, H, W, 3), device="cuda")
    with pytest.raises(fvv.FvvError) as e:
        it.run_batch(cams, [0, 1], np.array([0, 0, 0]), np.zeros(1, np.float32), out=dev_out)
    assert e.value.code == fvv.FVV_ESHAPE
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_interp_run(it.h, cams[0], cams[1], np.zeros(1, np.float32), 0, dev_out)
    assert e.value.code == fvv.FVV_ESHAPE
    fvv.fvv_interp_status(it.h)
    it.close()
    one.close()


def test_rig_instant_matches_oracle(torch_cuda):
    """A batched rig instant (4 pairs of a 5-camera arc, uneven view counts, random t)
    against the FP64 oracle, view by view, on the FP32 and the BF16 path."""
    torch = torch_cuda
    H, W = 48, 80
    frames = scene.rig(15, H, W, n_cams=5, max_disp=6.0)
    cams = [torch.from_numpy(c).cuda() for c in frames]
    rng = np.random.default_rng(15)
    counts = [2, 1, 3, 1]
    offs = np.concatenate([[0], np.cumsum(counts)])
    ts = np.concatenate([np.sort(rng.uniform(0, 1, c)) for c in counts]).astype(np.float32)
    refs = []
    for p in range(4):
        for v in range(offs[p], offs[p + 1]):
            refs.append(oracle.vinet_forward(blob(), frames[p], frames[p + 1], float(ts[v])))
    for precision in (fvv.FVV_FP32, fvv.FVV_BF16):
        it = fvv.Interpolator(blob(), H, W, precision=precision, max_views=8, max_cams=5)
        out = it.run_batch(cams, [0, 1, 2, 3], offs, ts).cpu().numpy()
        fvv.fvv_interp_status(it.h)
        for v, ref in enumerate(refs):
            if precision == fvv.FVV_FP32:
                err = float(np.abs(out[v] - ref).max())
                assert err <= 1e-4, (v, err)
            else:
                assert psnr(out[v], ref) >= 45.0, (v, psnr(out[v], ref))
        it.close()


@pytest.mark.parametrize("precision", [fvv.FVV_FP32, fvv.FVV_BF16])
def test_bucket_graphs_replay_any_view_mix(torch_cuda, precision):
    """Graphs are captured per view-count bucket (powers of two up to max_views), the
    kernels reading the call's counts from device memory: 24 rig instants with random
    per-pair counts (4..16 views) and single-pair calls of 1..16 views replay at most
    five graphs, and every output equals direct launches bit for bit."""
    torch = torch_cuda
    H, W = 48, 80
    cams = [torch.from_numpy(c).cuda() for c in scene.rig(16, H, W, n_cams=5, max_disp=6.0)]
    g = fvv.Interpolator(blob(), H, W, precision=precision, max_views=16, max_cams=5, graphs=1)
    d = fvv.Interpolator(blob(), H, W, precision=precision, max_views=16, max_cams=5, graphs=0)
    rng = np.random.default_rng(16)
    for _ in range(24):
        counts = rng.integers(1, 5, 4)
        offs = np.concatenate([[0], np.cumsum(counts)])
        ts = np.concatenate([np.sort(rng.uniform(0, 1, c)) for c in counts]).astype(np.float32)
        a = g.run_batch(cams, [0, 1, 2, 3], offs, ts).cpu().numpy()
        b = d.run_batch(cams, [0, 1, 2, 3], offs, ts).cpu().numpy()
        np.testing.assert_array_equal(a, b)
    for nv in (1, 3, 2, 16, 5, 9):
        ts = rng.uniform(0, 1, nv).astype(np.float32)
        a = g.run(cams[1], cams[2], ts).cpu().numpy()
        b = d.run(cams[1], cams[2], ts).cpu().numpy()
        np.testing.assert_array_equal(a, b)
    fvv.fvv_interp_status(g.h)
    assert g.graph_captures <= 5, g.graph_captures      # buckets 1, 2, 4, 8, 16
    assert d.graph_captures == 0


@pytest.mark.parametrize("precision", [fvv.FVV_FP32, fvv.FVV_BF16])
def test_contextnet_stream_fork_keeps_bits(torch_cuda, precision):
    torch = torch_cuda
    H, W = 136, 200
    left, right = pair(41, H, W, 7.0)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ts = [0.25, 0.75]
    for graphs in (1, 0):
        it = fvv.Interpolator(blob(), H, W, precision=precision, max_views=2, graphs=graphs)
        forked = it.run(L, R, ts).cpu().numpy()
        fvv.fvv_interp_profile(it.h, True)          # one stream, events around every conv
        serial = it.run(L, R, ts).cpu().numpy()
        fvv.fvv_interp_profile(it.h, False)
        again = it.run(L, R, ts).cpu().numpy()
        fvv.fvv_interp_status(it.h)
        np.testing.assert_array_equal(serial, forked)
        np.testing.assert_array_equal(again, forked)
        it.close()
