"""FP64 CPU oracle of the VINet forward (test infrastructure only).

Only tests, the smoke check and the bench's CPU-baseline leg may import this
package; the library's product path never does.  The arithmetic lives in
vinet_oracle.c (plain C, direct loops, OpenMP over output rows); this module
compiles it on demand and wraps it with numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vinet_oracle.c")
# two builds: AVX2/FMA hosts get the x86-64-v3 one, anything else the baseline one
_VARIANTS = {"v3": ["-march=x86-64-v3"], "base": []}
_lib = None


def _so(tag: str) -> str:
    return os.path.join(_HERE, f"liboracle_{tag}.so")


def build() -> None:
    """Compile every variant of the oracle library if it is missing or stale."""
    for tag, flags in _VARIANTS.items():
        so = _so(tag)
        if os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(_SRC):
            continue
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", *flags,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)


def _host_has_v3() -> bool:
    try:
        flags = open("/proc/cpuinfo").read()
    except OSError:
        return False
    return all(f" {f}" in flags for f in ("avx2", "fma", "bmi2"))


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_so("v3" if _host_has_v3() else "base"))
        D, I, F = ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(ctypes.c_float)
        L.oracle_conv3x3.argtypes = [D, I, I, I, F, F, I, I, I, I, D]
        L.oracle_convT.argtypes = [D, I, I, I, F, F, I, I, I, D]
        L.oracle_box_down.argtypes = [D, I, I, I, I, D]
        L.oracle_upsample2x.argtypes = [D, I, I, I, I, D]
        L.oracle_warp.argtypes = [D, I, I, I, D, I, I, D]
        L.oracle_blend.argtypes = [D, D, D, ctypes.c_long, I, D]
        L.oracle_n_floats.restype = ctypes.c_long
        L.oracle_layer_info.restype = ctypes.c_char_p
        L.oracle_layer_info.argtypes = [I] + [ctypes.POINTER(ctypes.c_int)] * 5
        L.oracle_vinet_forward.argtypes = [F, ctypes.c_long, F, F, I, I, ctypes.c_double, I, D,
                                           ctypes.c_void_p]
        L.oracle_lap_loss.argtypes = [D, D, I, I, I, I, D]
        L.oracle_lap_loss.restype = ctypes.c_double
        L.oracle_lap_down.argtypes = [D, I, I, I, D]
        L.oracle_lap_up.argtypes = [D, I, I, I, I, I, D]
        L.oracle_lap_levels.argtypes = [D, I, I, I, I, D]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def threads() -> int:
    return lib().oracle_threads()


def n_floats() -> int:
    return lib().oracle_n_floats()


def layer_table():
    """[(name, kind, C_in, C_out, stride, relu)] as the oracle reads the blob."""
    L = lib()
    out = []
    for i in range(L.oracle_n_layers()):
        v = [ctypes.c_int() for _ in range(5)]
        name = L.oracle_layer_info(i, *[ctypes.byref(x) for x in v])
        k, ci, co, s, r = (x.value for x in v)
        out.append((name.decode(), "conv" if k == 0 else "convT", ci, co, s, bool(r)))
    return out


def conv3x3(x, w, b, stride=1, circ=False, relu=False):
    """x: H x W x Ci; w: [Co][Ci][3][3]; returns Ho x Wo x Co (float64)."""
    x, w, b = _c64(x), _c32(w), _c32(b)
    H, W, Ci = x.shape
    Co = w.shape[0]
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    out = np.empty((Ho, Wo, Co))
    lib().oracle_conv3x3(_d(x), H, W, Ci, _f(w), _f(b), Co, stride, int(circ), int(relu), _d(out))
    return out


def conv_transpose4x4(x, w, b, circ=False, relu=False):
    """x: H x W x Ci; w: [Ci][Co][4][4]; stride 2, pad 1; returns 2H x 2W x Co."""
    x, w, b = _c64(x), _c32(w), _c32(b)
    H, W, Ci = x.shape
    Co = w.shape[1]
    out = np.empty((2 * H, 2 * W, Co))
    lib().oracle_convT(_d(x), H, W, Ci, _f(w), _f(b), Co, int(circ), int(relu), _d(out))
    return out


def box_down(x, f):
    x = _c64(x)
    H, W, C = x.shape
    out = np.empty((H // f, W // f, C))
    lib().oracle_box_down(_d(x), H, W, C, f, _d(out))
    return out


def upsample2x(x, circ=False):
    x = _c64(x)
    H, W, C = x.shape
    out = np.empty((2 * H, 2 * W, C))
    lib().oracle_upsample2x(_d(x), H, W, C, int(circ), _d(out))
    return out


def warp(img, flow, circ=False):
    """img: H x W x C; flow: H x W x 2 (F_x, F_y) in pixels; backward bilinear warp."""
    img, flow = _c64(img), _c64(flow)
    H, W, C = img.shape
    out = np.empty_like(img)
    lib().oracle_warp(_d(img), H, W, C, _d(flow), flow.shape[2], int(circ), _d(out))
    return out


def blend(a, b, M):
    a, b, M = _c64(a), _c64(b), _c64(M)
    out = np.empty_like(a)
    lib().oracle_blend(_d(a), _d(b), _d(M), M.size, a.shape[-1], _d(out))
    return out


class _Dumps(ctypes.Structure):
    _fields_ = [("vib_out", ctypes.c_void_p * 3), ("blend", ctypes.c_void_p), ("z", ctypes.c_void_p)]


def vinet_forward(blob, left, right, t, circ=False, dumps=False):
    """Full forward for one view.  left/right: H x W x 3 float32 in [0, 1].

    Returns the H x W x 3 float64 view, or (view, dict) with the intermediates
    'vib0'/'vib1'/'vib2' (stage flows + mask logit), 'blend' and 'z' (padded size).
    """
    blob, left, right = _c32(blob), _c32(left), _c32(right)
    H, W, _ = left.shape
    out = np.empty((H, W, 3))
    d = None
    arrs = {}
    if dumps:
        Hp, Wp = (H + 15) // 16 * 16, (W + 15) // 16 * 16
        for s in range(3):
            f = 2 ** (2 - s)
            arrs[f"vib{s}"] = np.empty((Hp // f, Wp // f, 5))
        arrs["blend"] = np.empty((Hp, Wp, 3))
        arrs["z"] = np.empty((Hp, Wp, 3))
        d = _Dumps()
        for s in range(3):
            d.vib_out[s] = arrs[f"vib{s}"].ctypes.data
        d.blend = arrs["blend"].ctypes.data
        d.z = arrs["z"].ctypes.data
    rc = lib().oracle_vinet_forward(_f(blob), blob.size, _f(left), _f(right), H, W, float(t),
                                    int(circ), _d(out), ctypes.byref(d) if d is not None else None)
    if rc != 0:
        raise ValueError(f"oracle_vinet_forward failed ({rc})")
    return (out, arrs) if dumps else out


def stitch_cluster(center, side_views, scale):
    """Multi-view cluster frame (Sec. 3.2, multiview organizer), in float64.

    The centre camera's real view at full resolution on top; below it the 2 x n_side
    views of its neighbourhood in arc order, each reduced by the scale x scale box
    average (the pyramid's box filter) and placed `scale` per row, row by row;
    unused tiles are zero.  The paper fixes the idea, not the layout: this layout is
    our reading.
    """
    c = np.asarray(center, np.float64)
    H, W, _ = c.shape
    n = len(side_views)
    th, tw = H // scale, W // scale
    rows = -(-n // scale)
    out = np.zeros((H + rows * th, W, 3))
    out[:H] = c
    for k, v in enumerate(side_views):
        small = np.asarray(v, np.float64).reshape(th, scale, tw, scale, 3).mean(axis=(1, 3))
        r, q = divmod(k, scale)
        out[H + r * th:H + (r + 1) * th, q * tw:(q + 1) * tw] = small
    return out


def lap_down(g):
    """One reduction step of the Laplace pyramid of Eq. 3: binomial [1 4 6 4 1]/16
    blur (edges replicated) sampled at even pixels; H x W x C -> ceil(H/2) x ceil(W/2) x C."""
    g = _c64(g)
    H, W, C = g.shape
    out = np.empty(((H + 1) // 2, (W + 1) // 2, C))
    lib().oracle_lap_down(_d(g), H, W, C, _d(out))
    return out


def lap_up(g, H, W):
    """One expansion step: the zero-inserted image filtered by 4 k k^T, at size H x W."""
    g = _c64(g)
    h, w, C = g.shape
    out = np.empty((H, W, C))
    lib().oracle_lap_up(_d(g), h, w, C, H, W, _d(out))
    return out


def lap_levels(img, levels=5):
    """[L^1, ..., L^levels] of one H x W x C image (L^levels = the last G)."""
    img = _c64(img)
    H, W, C = img.shape
    sizes = []
    h, w = H, W
    for _ in range(levels):
        sizes.append((h, w))
        h, w = (h + 1) // 2, (w + 1) // 2
    out = np.empty(sum(a * b for a, b in sizes) * C)
    lib().oracle_lap_levels(_d(img), H, W, C, levels, _d(out))
    res, off = [], 0
    for a, b in sizes:
        res.append(out[off:off + a * b * C].reshape(a, b, C))
        off += a * b * C
    return res


def lap_loss(pred, gt, levels=5):
    """Laplacian-pyramid loss of Eq. 3 (Sec. 3.1) for one image pair, in float64:
    sum_i 2^(i-1) || L^i(pred) - L^i(gt) ||_1 (L1 = sum over pixels and channels).
    Returns (loss, [norm of level 1, ..., norm of level `levels`])."""
    a, b = _c64(pred), _c64(gt)
    H, W, C = a.shape
    norms = np.empty(levels)
    loss = lib().oracle_lap_loss(_d(a), _d(b), H, W, C, levels, _d(norms))
    return float(loss), norms
