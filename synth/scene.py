"""Seeded synthetic layered-plane scenes (stand-in for the paper's 12-camera captures).

The paper evaluates on its own multi-camera recordings (Sec. 4.1) and Vimeo90K,
neither of which is available; these generated views have the same structure:
adjacent cameras on a horizontal baseline or arc, 3 textured fronto-parallel
planes at depths in [2, 10] (a full-frame backdrop at the largest depth, two
nearer rectangles that occlude it), so that the disparity between neighbours
spans a stated pixel range.

Recipe (all draws from numpy PCG64(seed), in the order written here):
* depths: z_near ~ U(2, 3), z_mid ~ U(3.5, 6), z_back ~ U(8, 10);
* near/mid rectangles: centre (x, y) ~ U(-0.25, 0.25) * frame half-extent at that
  depth, half-size ~ U(0.2, 0.35) / U(0.3, 0.45) of the frame width at that depth;
* textures: per plane and colour channel an independent permutation of 0..255
  driving 2-D gradient noise with the quintic fade 6t^5 - 15t^4 + 10t^3, summed
  over 4 octaves with persistence 0.5 (normalised), mapped 0.5 + 1.5 n and
  clamped to [0, 1]; base frequency 10 / z cycles per world unit, so features
  are of similar pixel size on every plane;  texture coordinates are world
  (X, Y) on the plane, so parallax is exact;
* pinhole camera, horizontal field of view 60 deg, principal point at the
  image centre, pixel (x, y) centred at (x + 0.5, y + 0.5); every pixel averages
  a 2x2 grid of rays at (+-0.25, +-0.25) px, each taking the colour of the
  nearest plane it hits.
* pair: cameras at X = -b/2 and +b/2 with f * b / 2 = max disparity (the
  disparity of a point at depth 2);
* rig: n cameras on a horizontal arc around (0, 0, 6) through the origin,
  each looking at that centre, the angular step chosen so that the disparity of
  the nearest depth (2) relative to the fixation depth is 0.9 * max disparity.

Outputs are float32 H x W x 3 (HWC) arrays in [0, 1].  The per-ray work runs in
the C helper render.c (compiled on first use), given the parameters drawn here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

FOV_DEG = 60.0
FIX_DEPTH = 6.0
CONTRAST = 1.5


_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib_handle = None


def build() -> str:
    """Compile the renderer helper (render.c) next to this file if it is stale."""
    src = os.path.join(_HERE, "render.c")
    if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        lib.synth_render.restype = None
        _lib_handle = lib
    return _lib_handle


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class Scene:
    """Three textured planes; the camera set is chosen by the caller."""

    def __init__(self, seed: int, W: int):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.f = 0.5 * W / np.tan(np.radians(FOV_DEG) / 2)
        zn, zm, zb = rng.uniform(2, 3), rng.uniform(3.5, 6), rng.uniform(8, 10)
        half_w = lambda z: 0.5 * W / self.f * z          # frame half-width at depth z
        self.planes = []
        for z, (lo, hi) in ((zn, (0.2, 0.35)), (zm, (0.3, 0.45))):
            cx, cy = rng.uniform(-0.25, 0.25, 2) * half_w(z)
            hs = rng.uniform(lo, hi) * 2 * half_w(z)
            self.planes.append((z, cx - hs, cx + hs, cy - hs, cy + hs))
        self.planes.append((zb, -1e9, 1e9, -1e9, 1e9))
        self.perms = []
        for _ in self.planes:
            ch = []
            for _ in range(3):
                p = rng.permutation(256)
                ch.append(np.concatenate([p, p]).astype(np.int32))
            self.perms.append(ch)
        self.offsets = rng.uniform(0, 64, (len(self.planes), 3, 2))

    def render(self, H: int, W: int, pos, yaw: float = 0.0) -> np.ndarray:
        """Image seen by a camera at world position pos, rotated by yaw about Y."""
        img = np.empty((H, W, 3), np.float32)
        planes = np.ascontiguousarray(np.array(self.planes, np.float64))
        perms = np.ascontiguousarray(np.stack([p for ch in self.perms for p in ch]).astype(np.int32))
        offs = np.ascontiguousarray(self.offsets.astype(np.float64))
        posa = np.array(pos, np.float64)
        _lib().synth_render(ctypes.c_int(H), ctypes.c_int(W), ctypes.c_double(self.f),
                            _ptr(posa, ctypes.c_double), ctypes.c_double(yaw),
                            ctypes.c_int(len(self.planes)), _ptr(planes, ctypes.c_double),
                            _ptr(perms, ctypes.c_int32), _ptr(offs, ctypes.c_double),
                            ctypes.c_double(CONTRAST), ctypes.c_int(4), ctypes.c_float(0.5),
                            _ptr(img, ctypes.c_float))
        return img


def stereo_pair(seed: int, H: int, W: int, max_disp: float):
    """(left, right) float32 HxWx3 views; disparity f*b/Z reaches max_disp at Z = 2."""
    sc = Scene(seed, W)
    b = 2.0 * max_disp / sc.f
    left = sc.render(H, W, (-b / 2, 0.0, 0.0))
    right = sc.render(H, W, (b / 2, 0.0, 0.0))
    return left, right


def stereo_views(seed: int, H: int, W: int, max_disp: float, ts):
    """(left, right, [view at t for t in ts]): the pair of stereo_pair and the same
    scene seen from the camera at X = -b/2 + t b between them (the ground truth a
    virtual view at t is compared with)."""
    sc = Scene(seed, W)
    b = 2.0 * max_disp / sc.f
    left = sc.render(H, W, (-b / 2, 0.0, 0.0))
    right = sc.render(H, W, (b / 2, 0.0, 0.0))
    mids = [sc.render(H, W, (-b / 2 + float(t) * b, 0.0, 0.0)) for t in ts]
    return left, right, mids


def rig(seed: int, H: int, W: int, n_cams: int = 9, max_disp: float = 64.0):
    """n_cams views on a horizontal arc fixating (0, 0, 6); list of HxWx3 arrays."""
    sc = Scene(seed, W)
    # relative disparity of depth 2 vs the fixation depth: f * B * (1/2 - 1/6)
    B = 0.9 * max_disp / (sc.f * (1.0 / 2.0 - 1.0 / FIX_DEPTH))
    dphi = B / FIX_DEPTH
    out = []
    for k in range(n_cams):
        phi = (k - (n_cams - 1) / 2.0) * dphi
        # camera k + 1 sits to the right (+X) of camera k and turns back to the centre
        pos = (FIX_DEPTH * np.sin(phi), 0.0, FIX_DEPTH - FIX_DEPTH * np.cos(phi))
        out.append(sc.render(H, W, pos, yaw=-phi))
    return out
