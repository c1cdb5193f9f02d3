"""Pins of the oracle's Laplacian-pyramid loss (Eq. 3, Sec. 3.1), CPU only.

The paper names a five-level Laplace pyramid and an L1 norm; the filter and the
borders are our reading (binomial [1 4 6 4 1]/16, replicated edges).  Each step of
the oracle is pinned to something other than itself:

* the reduction step against scipy's correlate (mode 'nearest' = replicated edges)
  of the separable kernel, sampled at even pixels;
* the expansion step against closed forms: a constant stays constant, a coarse
  delta becomes the 4 k k^T stencil centred on its fine pixel, a linear ramp
  sampled at the even pixels comes back as the ramp;
* the levels reassemble the image exactly (I = L1 + up(L2 + up(L3 + ...)));
* the loss of two constant images has a closed form (only L^5 differs);
* the loss depends only on the difference of the two images and is symmetric.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle

K = np.array([1, 4, 6, 4, 1], np.float64) / 16


@pytest.mark.parametrize("H,W", [(13, 18), (16, 16), (7, 5)])
def test_down_matches_library_correlate(H, W):
    g = np.random.default_rng(H * W).standard_normal((H, W, 2))
    ref = ndimage.correlate(g, np.outer(K, K)[..., None], mode="nearest")[::2, ::2]
    np.testing.assert_allclose(oracle.lap_down(g), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("H,W", [(13, 18), (16, 16), (9, 4)])
def test_up_keeps_constants(H, W):
    h, w = (H + 1) // 2, (W + 1) // 2
    g = np.full((h, w, 3), 0.37)
    np.testing.assert_allclose(oracle.lap_up(g, H, W), 0.37, rtol=0, atol=1e-15)


def test_up_of_delta_is_the_stencil():
    h, w = 8, 9
    g = np.zeros((h, w, 1))
    i, j = 3, 4
    g[i, j, 0] = 1.0
    up = oracle.lap_up(g, 2 * h, 2 * w)[..., 0]
    ref = np.zeros((2 * h, 2 * w))
    ref[2 * i - 2:2 * i + 3, 2 * j - 2:2 * j + 3] = 4 * np.outer(K, K)
    np.testing.assert_allclose(up, ref, rtol=0, atol=1e-15)


def test_up_interpolates_a_ramp():
    H, W = 12, 20
    fine = (3.0 * np.arange(W) + 1.0)[None, :, None] + 0.5 * np.arange(H)[:, None, None]
    coarse = fine[::2, ::2]
    up = oracle.lap_up(coarse, H, W)
    # away from the replicated edges the expansion reproduces a linear function
    np.testing.assert_allclose(up[2:-2, 2:-2], fine[2:-2, 2:-2], rtol=0, atol=1e-12)


@pytest.mark.parametrize("H,W", [(32, 48), (27, 35)])
def test_levels_reassemble_the_image(H, W):
    img = np.random.default_rng(5).random((H, W, 3))
    L = oracle.lap_levels(img, 5)
    rec = L[4]
    for i in (3, 2, 1, 0):
        rec = L[i] + oracle.lap_up(rec, *L[i].shape[:2])
    np.testing.assert_allclose(rec, img, rtol=0, atol=1e-12)
    # a constant image has no detail: L^1..L^4 vanish, L^5 is the constant
    Lc = oracle.lap_levels(np.full((H, W, 3), 0.6), 5)
    for i in range(4):
        assert np.abs(Lc[i]).max() < 1e-14
    np.testing.assert_allclose(Lc[4], 0.6, atol=1e-14)


def test_loss_of_constants_closed_form():
    H, W = 48, 80                       # level 5: 3 x 5 pixels
    a, b = np.full((H, W, 3), 0.75), np.full((H, W, 3), 0.25)
    loss, norms = oracle.lap_loss(a, b)
    assert norms[:4].max() < 1e-12
    np.testing.assert_allclose(norms[4], 0.5 * 3 * 5 * 3, rtol=1e-14)
    np.testing.assert_allclose(loss, 2 ** 4 * 0.5 * 3 * 5 * 3, rtol=1e-14)


def test_loss_depends_on_the_difference_only():
    rng = np.random.default_rng(9)
    a, b = rng.random((40, 56, 3)), rng.random((40, 56, 3))
    l_ab, n_ab = oracle.lap_loss(a, b)
    l_d, n_d = oracle.lap_loss(a - b, np.zeros_like(a))
    l_ba, _ = oracle.lap_loss(b, a)
    np.testing.assert_allclose(l_ab, l_d, rtol=1e-12)
    np.testing.assert_allclose(n_ab, n_d, rtol=1e-12)
    np.testing.assert_allclose(l_ab, l_ba, rtol=1e-14)
    np.testing.assert_allclose(l_ab, sum(2 ** i * n for i, n in enumerate(n_ab)), rtol=1e-14)
