"""GPU parity of the Laplacian-pyramid loss (Eq. 3) against the FP64 oracle.

fvv_lap_loss builds one pyramid of the difference pred - gt in FP32 (the pyramid is
linear) and sums each level's |.| in fixed order; the oracle builds both pyramids in
FP64 and subtracts level by level.  Bar, per level: every element of L^i comes out of
at most ~35 FP32 operations on values bounded by max |pred - gt|, so its error is
below 2e-6 max|D|; the level's norm may therefore differ by 2e-6 max|D| x (elements
of the level) plus the FP32 summation error (1e-5 of the norm).  The loss gets the same
bar through the level weights.

Cases: ragged and tiny sizes (odd sizes on every level, tiles cut by the image edge),
several pairs per call, two constant images (closed form), the bench's 1920 x 1080
configuration (two rendered views against the ground-truth view between them), a
second call giving the same bits, and argument checks.
"""
import numpy as np
import pytest

import oracle
import paper_2112_10603_b300 as fvv
from synth import scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    return torch


def _run(torch, pred, gt):
    n, H, W, _ = pred.shape
    ws_bytes = fvv.fvv_lap_loss_workspace(n, H, W)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    p = torch.from_numpy(np.ascontiguousarray(pred, np.float32)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(gt, np.float32)).cuda()
    loss = torch.empty(n, device="cuda")
    norms = torch.empty((n, 5), device="cuda")
    fvv.fvv_lap_loss(p, g, n, H, W, ws, ws_bytes, loss, norms)
    torch.cuda.synchronize()
    return loss.cpu().numpy(), norms.cpu().numpy()


def _check(pred, gt, loss, norms):
    for v in range(pred.shape[0]):
        ref, ref_n = oracle.lap_loss(pred[v].astype(np.float64), gt[v].astype(np.float64))
        dmax = float(np.abs(pred[v].astype(np.float64) - gt[v]).max())
        H, W = pred.shape[1:3]
        tot_tol = 0.0
        for i in range(5):
            count = H * W * 3
            tol = 2e-6 * dmax * count + 1e-5 * ref_n[i]
            assert abs(norms[v, i] - ref_n[i]) <= tol, (v, i, norms[v, i], ref_n[i], tol)
            tot_tol += 2 ** i * tol
            H, W = (H + 1) // 2, (W + 1) // 2
        assert abs(loss[v] - ref) <= tot_tol, (v, loss[v], ref, tot_tol)


@pytest.mark.parametrize("n,H,W", [(3, 37, 53), (2, 64, 96), (1, 130, 250), (2, 2, 2), (1, 3, 5), (1, 33, 65)])
def test_lap_loss_matches_oracle(torch_cuda, n, H, W):
    rng = np.random.default_rng(H * 1000 + W)
    pred = rng.random((n, H, W, 3)).astype(np.float32)
    gt = np.clip(pred + 0.1 * rng.standard_normal((n, H, W, 3)), 0, 1).astype(np.float32)
    loss, norms = _run(torch_cuda, pred, gt)
    _check(pred, gt, loss, norms)


def test_lap_loss_constants_closed_form(torch_cuda):
    H, W = 48, 80                       # level 5: 3 x 5 pixels
    pred = np.full((1, H, W, 3), 0.75, np.float32)
    gt = np.full((1, H, W, 3), 0.25, np.float32)
    loss, norms = _run(torch_cuda, pred, gt)
    assert np.abs(norms[0, :4]).max() < 1e-5
    np.testing.assert_allclose(norms[0, 4], 0.5 * 3 * 5 * 3, rtol=1e-6)
    np.testing.assert_allclose(loss[0], 16 * 0.5 * 3 * 5 * 3, rtol=1e-6)


def test_lap_loss_1080p_views_vs_ground_truth(torch_cuda):
    """The bench's configuration: 1920 x 1080 views against the rendered ground truth."""
    left, right, (mid,) = scene.stereo_views(2, 1080, 1920, 64.0, [0.5])
    pred = np.stack([left, right])
    gt = np.stack([mid, mid])
    loss, norms = _run(torch_cuda, pred, gt)
    _check(pred, gt, loss, norms)
    again = _run(torch_cuda, pred, gt)
    np.testing.assert_array_equal(again[0], loss)          # fixed-order sums: same bits
    np.testing.assert_array_equal(again[1], norms)


def test_lap_loss_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    x = torch.zeros((1, 8, 8, 3), device="cuda")
    out = torch.zeros(1, device="cuda")
    need = fvv.fvv_lap_loss_workspace(1, 8, 8)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_lap_loss(x, x, 1, 8, 8, ws, need - 1, out)
    assert e.value.code == fvv.FVV_EINVAL
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_lap_loss(x, x, 0, 8, 8, ws, need, out)
    assert e.value.code == fvv.FVV_ESHAPE
