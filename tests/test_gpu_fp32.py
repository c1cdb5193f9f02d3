"""GPU parity of the plain FP32 path (SIMT FFMA convolutions) against the FP64 oracle.

Bar: max |err| <= 1e-4 on output pixels in [0, 1], element by element, at sizes
that span several tiles and ragged tails; plus properties that hold exactly on
the FP32 path (batch invariance, circular shift equivariance).
"""
import numpy as np
import pytest

import paper_2112_10603_b300 as fvv
from tests.gpu_common import blob, oracle_view, pair

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    return torch


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _interp(H, W, **kw):
    return fvv.Interpolator(blob(), H, W, **kw)


def test_config1_256_fp32_matches_oracle(torch_cuda):
    torch = torch_cuda
    H = W = 256
    left, right = pair(1, H, W, 12.0)
    ref, dumps = oracle_view(1, H, W, 12.0, 0.5)
    it = _interp(H, W, max_views=1)
    out = it.run(_dev(torch, left), _dev(torch, right), [0.5]).cpu().numpy()[0]
    # stage by stage first, so that a failure names the stage
    for s in range(3):
        np.testing.assert_allclose(it.peek(f"vib{s}"), dumps[f"vib{s}"], atol=2e-4, rtol=1e-4,
                                   err_msg=f"stage {s} flows/mask")
    np.testing.assert_allclose(it.peek("blend"), dumps["blend"], atol=TOL, rtol=0)
    np.testing.assert_allclose(it.peek("z"), dumps["z"], atol=2e-4, rtol=1e-4)
    err = np.abs(out - ref).max()
    assert err <= TOL, err
    assert it.last_launches > 50


@pytest.mark.parametrize("H,W,ts", [(72, 100, (0.0, 0.3, 1.0)), (40, 200, (0.65,))])
def test_ragged_sizes_multi_view(torch_cuda, H, W, ts):
    torch = torch_cuda
    left, right = pair(5, H, W, 8.0)
    it = _interp(H, W, max_views=4)
    out = it.run(_dev(torch, left), _dev(torch, right), list(ts)).cpu().numpy()
    for k, t in enumerate(ts):
        ref, _ = oracle_view(5, H, W, 8.0, t)
        err = np.abs(out[k] - ref).max()
        assert err <= TOL, (t, err)


def test_circular_mode_and_shift_equivariance(torch_cuda):
    torch = torch_cuda
    H, W = 64, 96
    left, right = pair(6, H, W, 6.0)
    it = _interp(H, W, max_views=1, pad_mode=fvv.FVV_PAD_CIRCULAR)
    a = it.run(_dev(torch, left), _dev(torch, right), [0.5]).cpu().numpy()[0]
    ref, _ = oracle_view(6, H, W, 6.0, 0.5, circ=True)
    assert np.abs(a - ref).max() <= TOL
    sh = (16, -48)
    b = it.run(_dev(torch, np.roll(left, sh, (0, 1))), _dev(torch, np.roll(right, sh, (0, 1))), [0.5])
    np.testing.assert_array_equal(np.roll(a, sh, (0, 1)), b.cpu().numpy()[0])


def test_batch_invariance_and_host_path(torch_cuda):
    torch = torch_cuda
    H, W = 48, 80
    left, right = pair(7, H, W, 6.0)
    it = _interp(H, W, max_views=4)
    L, R = _dev(torch, left), _dev(torch, right)
    many = it.run(L, R, [0.2, 0.5, 0.9]).cpu().numpy()
    alone = it.run(L, R, [0.5]).cpu().numpy()
    np.testing.assert_array_equal(many[1], alone[0])
    host = it.run_host(left, right, [0.2, 0.5, 0.9])
    np.testing.assert_array_equal(host, many)


def test_pipelined_host_calls(torch_cuda):
    """Two host-buffer calls in flight (the copy-out of one overlapping the forward of
    the next), distinct inputs and view sets per call, pinned and pageable buffers: each
    call delivers exactly what the device-buffer call gives for its inputs."""
    torch = torch_cuda
    H, W = 48, 80
    it = _interp(H, W, max_views=3)
    calls = []
    for k in range(5):
        left, right = pair(30 + k, H, W, 6.0)
        ts = [0.1 * (k + 1), 0.95][: 1 + k % 2]
        if k % 2:
            lh, rh = torch.from_numpy(left).pin_memory(), torch.from_numpy(right).pin_memory()
            out = torch.full((len(ts), H, W, 3), -1.0).pin_memory()
        else:
            lh, rh, out = left, right, np.full((len(ts), H, W, 3), -1.0, np.float32)
        calls.append((left, right, ts, lh, rh, out))
    tickets = []
    for k, (_, _, ts, lh, rh, out) in enumerate(calls):
        tickets.append(it.submit_host(lh, rh, ts, out))
        if k:
            it.wait_host(tickets[k - 1])
    it.wait_host(tickets[-1])
    it.wait_host(tickets[0])          # long done: returns at once
    assert tickets == list(range(tickets[0], tickets[0] + 5))
    for left, right, ts, _, _, out in calls:
        want = it.run(_dev(torch, left), _dev(torch, right), ts).cpu().numpy()
        got = out.numpy() if hasattr(out, "numpy") else out
        np.testing.assert_array_equal(got, want)
    with pytest.raises(fvv.FvvError):
        it.wait_host(tickets[-1] + 1)
    fvv.fvv_interp_status(it.h)


def test_run_batch_matches_per_pair_runs(torch_cuda):
    torch = torch_cuda
    from synth import scene
    H, W = 48, 64
    cams = scene.rig(8, H, W, n_cams=3, max_disp=6.0)
    it = _interp(H, W, max_views=4, max_cams=3)
    dc = [_dev(torch, c) for c in cams]
    out = it.run_batch(dc, [0, 1], [0, 2, 3], [0.25, 0.75, 0.5]).cpu().numpy()
    single = _interp(H, W, max_views=2)
    a = single.run(dc[0], dc[1], [0.25, 0.75]).cpu().numpy()
    b = single.run(dc[1], dc[2], [0.5]).cpu().numpy()
    np.testing.assert_array_equal(out[:2], a)
    np.testing.assert_array_equal(out[2], b[0])


def test_argument_errors(torch_cuda):
    torch = torch_cuda
    it = _interp(32, 32, max_views=2)
    x = torch.zeros(32, 32, 3, device="cuda")
    out = torch.empty(3, 32, 32, 3, device="cuda")
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_interp_run(it.h, x, x, np.array([0.1, 0.2, 0.3], np.float32), 3, out)
    assert e.value.code == fvv.FVV_ESHAPE
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_interp_run(it.h, x, x, np.array([1.5], np.float32), 1, out)
    assert e.value.code == fvv.FVV_EINVAL
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_interp_run_batch(it.h, [x, x], [1], [0, 1], [0.5], out)
    assert e.value.code == fvv.FVV_EINVAL


def test_full_1080p_seven_views_fp32(torch_cuda):
    """The bench's workload (1920x1080, 7 views t = k/8) on the FP32 path: the
    midpoint view element-wise against the oracle, every view finite and in
    [0, 1], and each view equal to the same view computed alone."""
    torch = torch_cuda
    H, W = 1080, 1920
    left, right = pair(2, H, W, 64.0)
    ts = [k / 8 for k in range(1, 8)]
    it = _interp(H, W, max_views=7)
    L, R = _dev(torch, left), _dev(torch, right)
    out = it.run(L, R, ts).cpu().numpy()
    assert np.isfinite(out).all() and out.min() >= 0 and out.max() <= 1
    ref, _ = oracle_view(2, H, W, 64.0, 0.5)
    err = np.abs(out[3] - ref).max()
    assert err <= TOL, err
    alone = it.run(L, R, [ts[0]]).cpu().numpy()
    np.testing.assert_array_equal(alone[0], out[0])
