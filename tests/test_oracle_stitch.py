"""Pins of the oracle's multi-view cluster frame (Sec. 3.2, multiview organizer).

The cluster frame is a layout, so it is pinned by what it must contain: the centre
view unchanged, every tile equal to the oracle library's box filter (a separate
implementation, the C pyramid routine) of its view, tiles in arc order at their
places, empty tiles zero, and the paper's cluster size (16 views per side + the
centre = 33 views, Sec. 4.2)."""
import numpy as np

import oracle


def _views(rng, n, H, W):
    return [rng.uniform(0, 1, (H, W, 3)) for _ in range(n)]


def test_center_and_tiles_match_the_box_filter():
    rng = np.random.default_rng(0)
    H, W, s = 24, 40, 4
    center = rng.uniform(0, 1, (H, W, 3))
    side = _views(rng, 6, H, W)
    out = oracle.stitch_cluster(center, side, s)
    assert out.shape == (H + 2 * (H // s), W, 3)
    np.testing.assert_array_equal(out[:H], center)
    th, tw = H // s, W // s
    for k, v in enumerate(side):
        r, q = divmod(k, s)
        tile = out[H + r * th:H + (r + 1) * th, q * tw:(q + 1) * tw]
        np.testing.assert_allclose(tile, oracle.box_down(v, s), rtol=0, atol=1e-12)
    # tiles 6 and 7 of the second row are unused
    assert (out[H + th:, 2 * tw:] == 0).all()


def test_tiles_in_arc_order():
    H, W, s = 16, 16, 2
    side = [np.full((H, W, 3), float(k + 1)) for k in range(8)]    # 2 x n_side, n_side = 4
    out = oracle.stitch_cluster(np.zeros((H, W, 3)), side, s)
    th, tw = H // s, W // s
    for k in range(8):
        r, q = divmod(k, s)
        assert (out[H + r * th:H + (r + 1) * th, q * tw:(q + 1) * tw] == k + 1).all()


def test_paper_cluster_size():
    # 16 views per side + the real view = 33 views per cluster; at scale 4 the 32
    # side tiles fill 8 rows of 4 below the real view: a W x 3H frame
    H, W = 32, 64
    side = [np.zeros((H, W, 3)) for _ in range(32)]
    out = oracle.stitch_cluster(np.ones((H, W, 3)), side, 4)
    assert out.shape == (3 * H, W, 3) and 1 + len(side) == 33
