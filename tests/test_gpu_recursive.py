"""Recursive (paper-faithful) dense views, FVV_T_RECURSIVE (Sec. 4.2, supplement S.3):
the view at t = k / 2^n is the midpoint view of its two dyadic neighbours.

* each returned view equals the midpoint network applied by hand to the images it
  depends on (bit for bit, same kernels);
* against the oracle composed the same way, max |err| <= 1e-4 (FP32 path);
* n stages give 2^n - 1 views (the paper: 3 stages -> 7, 4 stages -> 15);
* non-dyadic t is rejected."""
import numpy as np
import pytest

import oracle
import paper_2112_10603_b300 as fvv
from tests.gpu_common import blob, pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    return torch


@pytest.mark.parametrize("precision", [fvv.FVV_FP32, fvv.FVV_BF16])
def test_recursive_equals_stacked_midpoints(torch_cuda, precision):
    torch = torch_cuda
    H, W = 64, 96
    left, right = pair(30, H, W, 6.0)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    rec = fvv.Interpolator(blob(), H, W, precision=precision, max_views=4, t_mode=fvv.FVV_T_RECURSIVE)
    out = rec.run(L, R, [0.25, 0.5, 0.75, 0.375]).cpu().numpy()
    d = fvv.Interpolator(blob(), H, W, precision=precision, max_views=1)
    mid = d.run(L, R, [0.5]).clone()
    q1 = d.run(L, mid[0], [0.5]).clone()
    q3 = d.run(mid[0], R, [0.5]).clone()
    e3 = d.run(q1[0], mid[0], [0.5]).clone()          # 3/8 between 1/4 and 1/2
    np.testing.assert_array_equal(out[1], mid.cpu().numpy()[0])
    np.testing.assert_array_equal(out[0], q1.cpu().numpy()[0])
    np.testing.assert_array_equal(out[2], q3.cpu().numpy()[0])
    np.testing.assert_array_equal(out[3], e3.cpu().numpy()[0])


def test_recursive_vs_composed_oracle(torch_cuda):
    torch = torch_cuda
    H, W = 48, 80
    left, right = pair(31, H, W, 6.0)
    b = blob()
    m = oracle.vinet_forward(b, left, right, 0.5).astype(np.float32)
    q1 = oracle.vinet_forward(b, left, m, 0.5)
    rec = fvv.Interpolator(b, H, W, precision=fvv.FVV_FP32, max_views=2, t_mode=fvv.FVV_T_RECURSIVE)
    out = rec.run(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), [0.25, 0.5]).cpu().numpy()
    assert np.abs(out[1] - m).max() <= 1e-4
    assert np.abs(out[0] - q1).max() <= 1e-4


@pytest.mark.parametrize("stages", [3, 4])
def test_dyadic_view_count(torch_cuda, stages):
    torch = torch_cuda
    H, W = 32, 64
    left, right = pair(32, H, W, 4.0)
    n = 2 ** stages - 1
    ts = [k / 2 ** stages for k in range(1, n + 1)]
    rec = fvv.Interpolator(blob(), H, W, precision=fvv.FVV_BF16, max_views=n, t_mode=fvv.FVV_T_RECURSIVE)
    out = rec.run(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), ts).cpu().numpy()
    assert out.shape[0] == n == 2 ** stages - 1
    assert np.isfinite(out).all()
    # consecutive views differ (each is its own synthesis)
    assert all(np.abs(out[i] - out[i + 1]).max() > 0 for i in range(n - 1))
    with pytest.raises(fvv.FvvError) as e:
        rec.run(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), [0.3])
    assert e.value.code == fvv.FVV_EINVAL
