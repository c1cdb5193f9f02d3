"""GPU parity of the multi-view cluster frame kernel (fvv_stitch_cluster) against
the oracle: the centre region bit for bit, the tiles (FP32 box averages of 4 or 16
values) within 1e-6, empty tiles zero; argument errors."""
import numpy as np
import pytest

import oracle
import paper_2112_10603_b300 as fvv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    return torch


@pytest.mark.parametrize("H,W,n_side,scale", [(64, 96, 16, 4), (48, 80, 5, 4), (40, 72, 3, 2)])
def test_stitch_matches_oracle(torch_cuda, H, W, n_side, scale):
    torch = torch_cuda
    rng = np.random.default_rng(H + n_side)
    center = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    side = [rng.uniform(0, 1, (H, W, 3)).astype(np.float32) for _ in range(2 * n_side)]
    rows = -(-2 * n_side // scale)
    out = torch.full((H + rows * (H // scale), W, 3), -1.0, device="cuda")
    dc = torch.from_numpy(center).cuda()
    ds = [torch.from_numpy(v).cuda() for v in side]
    fvv.fvv_stitch_cluster(dc, ds, H, W, scale, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = oracle.stitch_cluster(center, side, scale)
    np.testing.assert_array_equal(got[:H], center)
    assert np.abs(got - ref).max() <= 1e-6


def test_stitch_argument_errors(torch_cuda):
    torch = torch_cuda
    x = torch.zeros(30, 40, 3, device="cuda")
    out = torch.zeros(60, 40, 3, device="cuda")
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_stitch_cluster(x, [x, x], 30, 40, 4, out)        # 4 does not divide 30
    assert e.value.code == fvv.FVV_ESHAPE
    with pytest.raises(ValueError):
        fvv.fvv_stitch_cluster(x, [x], 30, 40, 2, out)            # odd number of side views
