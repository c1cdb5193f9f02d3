"""The server on the GPU: every result of a mixed-resolution, mixed-pair request mix
equals the same view computed alone by an interpolator (bit for bit: the batch is
one forward over independent views, and each output element's arithmetic does not
depend on its neighbours in the batch), and matches the FP64 oracle's view of the
same pair and t (BF16: PSNR >= 45 dB).  In dense mode the served views are those of
the snapped t = k / 2^n, again against the interpolator alone and the oracle."""
import ctypes
import time

import numpy as np
import pytest

import oracle
import paper_2112_10603_b300 as fvv
from synth import scene
from tests.gpu_common import blob, psnr

pytestmark = pytest.mark.gpu


def _fetch(ptr, shape):
    """Host copy of a device buffer the server owns (test helper)."""
    out = np.empty(shape, np.float32)
    rt = ctypes.CDLL("libcudart.so.13")
    rc = rt.cudaMemcpy(ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(ptr), ctypes.c_size_t(out.nbytes), 2)
    assert rc == 0
    return out


def test_server_mix_matches_alone():
    import torch
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    sizes = [(48, 80), (64, 96)]
    frames = {r: scene.rig(20 + r, h, w, n_cams=3, max_disp=6.0) for r, (h, w) in enumerate(sizes)}
    cams = {r: [torch.from_numpy(c).cuda() for c in frames[r]] for r in frames}
    cfg = fvv.fvv_serve_default_cfg(precision=fvv.FVV_BF16, n_res=2, res_h=[h for h, _ in sizes],
                                    res_w=[w for _, w in sizes], n_cams=3, slots_per_res=2, max_batch=3,
                                    pool_views=16)
    s = fvv.fvv_serve_create(blob(), cfg)
    try:
        for r in range(2):
            fvv.fvv_serve_set_frames(s, 0, r, cams[r])
        rng = np.random.default_rng(3)
        reqs = []
        for u in range(10):
            r, p, t = int(rng.integers(0, 2)), int(rng.integers(0, 2)), float(rng.uniform(0, 1))
            reqs.append((fvv.fvv_serve_submit(s, u, p, t, r), r, p, t))
            time.sleep(0.002 * (u % 3))          # arrivals spread over several batches
        alone = {r: fvv.Interpolator(blob(), h, w, precision=fvv.FVV_BF16, max_views=1)
                 for r, (h, w) in enumerate(sizes)}
        for tk, r, p, t in reqs:
            t0 = time.time()
            while True:
                st, ptr, lat = fvv.fvv_serve_poll(s, tk)
                if st == 0:
                    break
                assert time.time() - t0 < 30
                time.sleep(0.001)
            h, w = sizes[r]
            got = _fetch(ptr, (h, w, 3))
            ref = alone[r].run(cams[r][p], cams[r][p + 1], [t]).cpu().numpy()[0]
            np.testing.assert_array_equal(got, ref)
            ref64 = oracle.vinet_forward(blob(), frames[r][p], frames[r][p + 1], t)
            assert psnr(got, ref64) >= 45.0, (r, p, t, psnr(got, ref64))
            assert lat > 0
            assert fvv.fvv_serve_release(s, tk) == 0
        st = fvv.fvv_serve_stats_get(s)
        assert st["completed"] == 10 and st["failed"] == 0 and st["device_bytes"] > 0
    finally:
        fvv.fvv_serve_destroy(s)


def test_dense_mode_views_match_alone():
    """Dense mode: the per-instant view set, served by snapping t to k / 2^n, equals
    each view computed alone at t = k / 2^n (bit for bit); a new instant's frames
    give that instant's views."""
    import torch
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    h, w = 48, 80
    frames_np = [scene.rig(30 + i, h, w, n_cams=3, max_disp=6.0) for i in range(2)]
    frames = [[torch.from_numpy(c).cuda() for c in f] for f in frames_np]
    cfg = fvv.fvv_serve_default_cfg(precision=fvv.FVV_BF16, n_res=1, res_h=[h], res_w=[w], n_cams=3,
                                    slots_per_res=2, max_batch=6, dense_levels=2)
    s = fvv.fvv_serve_create(blob(), cfg)
    alone = fvv.Interpolator(blob(), h, w, precision=fvv.FVV_BF16, max_views=1)
    try:
        for inst in range(2):
            cams = frames[inst]
            fvv.fvv_serve_set_frames(s, inst, 0, cams)
            for u, (p, t) in enumerate([(0, 0.3), (1, 0.5), (0, 0.8), (1, 0.05), (0, 0.97)]):
                tk = fvv.fvv_serve_submit(s, 10 * inst + u, p, t, 0)
                t0 = time.time()
                while True:
                    st, ptr, lat = fvv.fvv_serve_poll(s, tk)
                    if st == 0:
                        break
                    assert time.time() - t0 < 30
                    time.sleep(0.001)
                got = _fetch(ptr, (h, w, 3))
                k = min(4, max(0, round(t * 4)))
                if k in (0, 4):
                    ref = cams[p if k == 0 else p + 1].cpu().numpy()
                else:
                    ref = alone.run(cams[p], cams[p + 1], [k / 4]).cpu().numpy()[0]
                    ref64 = oracle.vinet_forward(blob(), frames_np[inst][p], frames_np[inst][p + 1], k / 4)
                    assert psnr(got, ref64) >= 45.0, (inst, p, t, psnr(got, ref64))
                np.testing.assert_array_equal(got, ref)
                fvv.fvv_serve_release(s, tk)
            st = fvv.fvv_serve_stats_get(s)
            assert st["dense_instants"] == inst + 1 and st["failed"] == 0
    finally:
        fvv.fvv_serve_destroy(s)


def test_dense_immediate_fp8_views_match_alone_and_oracle():
    """FP8 dense server with immediate answers (3 levels, 7 views per pair): after the
    first set has rendered, requests are answered at once; every answered view equals
    the same view of an FP8 interpolator calibrated on the same frames (bit for bit),
    and is held to the FP8 floor of the small-size tests against the oracle."""
    import torch
    from paper_2112_10603_b300 import build as fvv_build
    fvv_build.build()
    h, w = 48, 80
    frames_np = scene.rig(40, h, w, n_cams=3, max_disp=6.0)
    cams = [torch.from_numpy(c).cuda() for c in frames_np]
    cal = []
    for sd in (100, 101):
        cal += list(scene.stereo_pair(sd, h, w, 6.0))
    cal_d = torch.from_numpy(np.stack(cal)).cuda()
    cfg = fvv.fvv_serve_default_cfg(precision=fvv.FVV_FP8, n_res=1, res_h=[h], res_w=[w], n_cams=3,
                                    slots_per_res=2, max_batch=14, dense_levels=3, dense_immediate=1)
    s = fvv.fvv_serve_create(blob(), cfg)
    alone = fvv.Interpolator(blob(), h, w, precision=fvv.FVV_FP8, max_views=1)
    fvv.fvv_calibrate_fp8(alone.h, cal_d, 2)
    try:
        fvv.fvv_serve_calibrate_fp8(s, 0, cal_d, 2)
        fvv.fvv_serve_set_frames(s, 0, 0, cams)
        t0 = time.time()
        while fvv.fvv_serve_stats_get(s)["dense_instants"] < 1:
            assert time.time() - t0 < 60
            time.sleep(0.002)
        for u, (p, t) in enumerate([(0, 0.3), (1, 0.5), (0, 0.88), (1, 0.12)]):
            tk = fvv.fvv_serve_submit(s, u, p, t, 0)
            st, ptr, lat = fvv.fvv_serve_poll(s, tk)
            assert st == 0                                   # answered at submit
            got = _fetch(ptr, (h, w, 3))
            k = min(8, max(0, round(t * 8)))
            ref = alone.run(cams[p], cams[p + 1], [k / 8]).cpu().numpy()[0]
            np.testing.assert_array_equal(got, ref)
            ref64 = oracle.vinet_forward(blob(), frames_np[p], frames_np[p + 1], k / 8)
            assert psnr(got, ref64) >= 30.0, (p, t, psnr(got, ref64))
            fvv.fvv_serve_release(s, tk)
        st = fvv.fvv_serve_stats_get(s)
        assert st["failed"] == 0 and st["stale_max"] == 0
    finally:
        fvv.fvv_serve_destroy(s)
