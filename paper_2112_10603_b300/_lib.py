"""ctypes binding of libfvv.so: the C ABI with the same names, arguments marshalled.

Device buffers may be given as torch CUDA tensors (their data_ptr is passed) or
as raw integer addresses; host buffers as numpy arrays.  Streams are torch
streams, raw cudaStream_t integers, or None (torch's current stream).
Every step of the computation runs in libfvv.so; there is no other path, and
loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfvv.so")

FVV_OK, FVV_EINVAL, FVV_ESHAPE, FVV_ENOMEM, FVV_ECUDA, FVV_EBUSY, FVV_ETIMEOUT, FVV_ESUPERSEDED, \
    FVV_ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7, -8
FVV_FP32, FVV_BF16, FVV_FP8 = 0, 1, 2
FVV_PAD_ZERO, FVV_PAD_CIRCULAR = 0, 1
FVV_T_DIRECT, FVV_T_RECURSIVE = 0, 1

ERROR_NAMES = {0: "FVV_OK", -1: "FVV_EINVAL", -2: "FVV_ESHAPE", -3: "FVV_ENOMEM", -4: "FVV_ECUDA",
               -5: "FVV_EBUSY", -6: "FVV_ETIMEOUT", -7: "FVV_ESUPERSEDED", -8: "FVV_ENOTFOUND"}


class FvvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class fvv_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("pad_mode", ctypes.c_int), ("t_mode", ctypes.c_int),
                ("max_views", ctypes.c_int), ("max_cams", ctypes.c_int), ("graphs", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p


def lib():
    """The loaded libfvv.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfvv.so not built at {LIB_PATH}; run paper_2112_10603_b300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.fvv_last_error.restype = ctypes.c_char_p
        L.fvv_default_opts.argtypes = [ctypes.POINTER(fvv_opts)]
        L.fvv_interp_create.argtypes = [_P, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(fvv_opts), ctypes.POINTER(_P)]
        L.fvv_interp_run.argtypes = [_P, _P, _P, _P, ctypes.c_int, _P, _P]
        L.fvv_interp_run_host.argtypes = [_P, _P, _P, _P, ctypes.c_int, _P, _P]
        L.fvv_interp_submit_host.argtypes = [_P, _P, _P, _P, ctypes.c_int, _P, _P,
                                             ctypes.POINTER(ctypes.c_longlong)]
        L.fvv_interp_wait_host.argtypes = [_P, ctypes.c_longlong]
        L.fvv_interp_run_batch.argtypes = [_P, _P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, _P]
        L.fvv_interp_device_bytes.argtypes = [_P]
        L.fvv_interp_device_bytes.restype = ctypes.c_size_t
        L.fvv_interp_last_launches.argtypes = [_P]
        L.fvv_interp_graph_captures.argtypes = [_P]
        L.fvv_interp_graph_captures.restype = ctypes.c_longlong
        L.fvv_interp_peek.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t]
        L.fvv_interp_layer.argtypes = [_P, ctypes.c_int, _P] + [ctypes.c_int] * 5 + [_P] + [ctypes.c_int] * 3 + [_P]
        L.fvv_interp_status.argtypes = [_P]
        L.fvv_interp_inject_stall.argtypes = [_P, ctypes.c_longlong]
        L.fvv_lap_loss_workspace.argtypes = [ctypes.c_int] * 3
        L.fvv_lap_loss_workspace.restype = ctypes.c_size_t
        L.fvv_lap_loss.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t, _P, _P, _P]
        L.fvv_interp_autotune.argtypes = [_P, ctypes.c_int, ctypes.c_char_p]
        L.fvv_layer_noalloc.argtypes = [ctypes.c_int, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P]
        L.fvv_interp_profile.argtypes = [_P, ctypes.c_int]
        L.fvv_stitch_cluster.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]
        L.fvv_interp_layer_stats.argtypes = [_P, _P, _P, _P, ctypes.c_int]
        L.fvv_interp_destroy.argtypes = [_P]
        _lib = L
    return _lib


def _check(rc: int):
    if rc != FVV_OK:
        raise FvvError(rc, lib().fvv_last_error().decode())


def _dev(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError(f"cannot take a device address from {type(x)}")


def _stream(s) -> int:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _host_f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data


def fvv_default_opts(**kw) -> fvv_opts:
    o = fvv_opts()
    lib().fvv_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def fvv_interp_create(weights, H: int, W: int, opts: fvv_opts | None = None) -> int:
    w, wp = _host_f32(weights)
    h = _P()
    _check(lib().fvv_interp_create(wp, w.size, H, W, ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(h)))
    return h.value


def fvv_interp_run(h: int, left, right, t, n_views: int, out, stream=None):
    ta, tp = _host_f32(t)
    _check(lib().fvv_interp_run(h, _dev(left), _dev(right), tp, n_views, _dev(out), _stream(stream)))


def _host_buf(a, writable=False):
    """(keepalive, address) of a host float32 buffer: numpy array or CPU torch tensor
    (a pinned tensor keeps its page-locked address)."""
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous() or str(a.dtype) != "torch.float32":
            raise ValueError("expected a contiguous float32 CPU tensor")
        return a, a.data_ptr()
    if writable:
        if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous):
            raise ValueError("out must be a C-contiguous float32 numpy array")
        return a, a.ctypes.data
    return _host_f32(a)


def fvv_interp_run_host(h: int, left, right, t, n_views: int, out, stream=None):
    la, lp = _host_buf(left)
    ra, rp = _host_buf(right)
    ta, tp = _host_f32(t)
    oa, op = _host_buf(out, writable=True)
    _check(lib().fvv_interp_run_host(h, lp, rp, tp, n_views, op, _stream(stream)))


def fvv_interp_submit_host(h: int, left, right, t, n_views: int, out, stream=None) -> int:
    """Enqueue a host-buffer call and return its ticket.  The copies run after this
    returns, so left, right and out are used in place (float32, C-contiguous; no
    temporary copy is made) and must stay alive until fvv_interp_wait_host."""
    _, lp = _host_buf(left, writable=True)
    _, rp = _host_buf(right, writable=True)
    ta, tp = _host_f32(t)
    _, op = _host_buf(out, writable=True)
    tk = ctypes.c_longlong(-1)
    _check(lib().fvv_interp_submit_host(h, lp, rp, tp, n_views, op, _stream(stream), ctypes.byref(tk)))
    return tk.value


def fvv_interp_wait_host(h: int, ticket: int):
    _check(lib().fvv_interp_wait_host(h, ticket))


def fvv_interp_run_batch(h: int, cams, pair_left, view_offsets, t, out, stream=None):
    ptrs = (ctypes.c_void_p * len(cams))(*[_dev(c) for c in cams])
    pl = np.ascontiguousarray(pair_left, dtype=np.int32)
    vo = np.ascontiguousarray(view_offsets, dtype=np.int32)
    ta, tp = _host_f32(t)
    _check(lib().fvv_interp_run_batch(h, ptrs, len(cams), pl.ctypes.data, vo.ctypes.data, tp, len(pl),
                                      _dev(out), _stream(stream)))


def fvv_interp_device_bytes(h: int) -> int:
    return lib().fvv_interp_device_bytes(h)


def fvv_interp_last_launches(h: int) -> int:
    return lib().fvv_interp_last_launches(h)


def fvv_interp_graph_captures(h: int) -> int:
    return int(lib().fvv_interp_graph_captures(h))


def fvv_interp_peek(h: int, which: int, view: int, shape):
    """Host copy (numpy float32, given shape) of an intermediate of the last run."""
    out = np.empty(shape, np.float32)
    _check(lib().fvv_interp_peek(h, which, view, out.ctypes.data, out.size))
    return out


def fvv_interp_layer(h: int, layer: int, inp, in_cs: int, in_coff: int, n: int, H: int, W: int,
                     out, out_cs: int, out_coff: int, out_f32: bool, stream=None):
    _check(lib().fvv_interp_layer(h, layer, _dev(inp), in_cs, in_coff, n, H, W, _dev(out), out_cs, out_coff,
                                  int(out_f32), _stream(stream)))


def fvv_layer_noalloc(layer: int, w, b, inp, in_cs: int, in_coff: int, n: int, H: int, W: int,
                      out, out_cs: int, out_coff: int, stream=None):
    """One layer with the caller's device weights and no device allocation (see fvv.h)."""
    _check(lib().fvv_layer_noalloc(layer, _dev(w), _dev(b), _dev(inp), in_cs, in_coff, n, H, W, _dev(out),
                                   out_cs, out_coff, _stream(stream)))


def fvv_stitch_cluster(center, side_views, H: int, W: int, scale: int, out, stream=None):
    """Cluster frame of one camera: centre view + 2 x n_side downscaled arc views (see fvv.h)."""
    ptrs = (ctypes.c_void_p * len(side_views))(*[_dev(v) for v in side_views])
    if len(side_views) % 2:
        raise ValueError("side_views must hold 2 x n_side views")
    _check(lib().fvv_stitch_cluster(_dev(center), ptrs, len(side_views) // 2, H, W, scale, _dev(out),
                                    _stream(stream)))


def fvv_interp_autotune(h: int, n_views: int, cache_path: str | None = None):
    _check(lib().fvv_interp_autotune(h, n_views, cache_path.encode() if cache_path else None))


def fvv_interp_status(h: int):
    _check(lib().fvv_interp_status(h))


def fvv_lap_loss_workspace(n: int, H: int, W: int) -> int:
    return int(lib().fvv_lap_loss_workspace(n, H, W))


def fvv_lap_loss(pred, gt, n: int, H: int, W: int, workspace, workspace_bytes: int, loss, level_norms=None,
                 stream=None):
    """Laplacian-pyramid loss of Eq. 3 for n image pairs (device buffers, see fvv.h)."""
    _check(lib().fvv_lap_loss(_dev(pred), _dev(gt), n, H, W, _dev(workspace), workspace_bytes, _dev(loss),
                              _dev(level_norms), _stream(stream)))


def fvv_interp_inject_stall(h: int, cycles: int):
    """Arm the next fvv_interp_layer call's bounded-wait fault injection (see fvv.h)."""
    _check(lib().fvv_interp_inject_stall(h, cycles))


def fvv_interp_profile(h: int, enable: bool):
    _check(lib().fvv_interp_profile(h, int(enable)))


N_LAYERS = 51


def fvv_interp_layer_stats(h: int):
    """(ms, flops, launches) arrays of length 51 since the last reset."""
    ms = np.zeros(N_LAYERS)
    fl = np.zeros(N_LAYERS)
    ln = np.zeros(N_LAYERS, np.int32)
    _check(lib().fvv_interp_layer_stats(h, ms.ctypes.data, fl.ctypes.data, ln.ctypes.data, N_LAYERS))
    return ms, fl, ln


def fvv_interp_destroy(h: int):
    lib().fvv_interp_destroy(h)


def fvv_last_error() -> str:
    return lib().fvv_last_error().decode()


# ---------------------------------------------------------------------------
# server

FVV_SERVE_MAX_RES = 4


class fvv_serve_cfg(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("n_res", ctypes.c_int),
                ("res_h", ctypes.c_int * FVV_SERVE_MAX_RES), ("res_w", ctypes.c_int * FVV_SERVE_MAX_RES),
                ("n_cams", ctypes.c_int), ("slots_per_res", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("pool_views", ctypes.c_int), ("hbm_budget", ctypes.c_size_t), ("fake_ms_per_view", ctypes.c_double),
                ("dense_levels", ctypes.c_int), ("dense_immediate", ctypes.c_int)]


class fvv_serve_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_longlong) for n in ("submitted", "completed", "superseded", "rejected", "failed",
                                                   "batches", "batched_views", "queued")] + \
               [("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("dense_instants", ctypes.c_longlong),
                ("age_p50_ms", ctypes.c_double), ("age_p99_ms", ctypes.c_double), ("stale_mean", ctypes.c_double),
                ("stale_max", ctypes.c_longlong)]


def _serve_sigs(L):
    if getattr(L, "_serve_ready", False):
        return L
    L.fvv_serve_default_cfg.argtypes = [ctypes.POINTER(fvv_serve_cfg)]
    L.fvv_serve_create.argtypes = [_P, ctypes.c_size_t, ctypes.POINTER(fvv_serve_cfg), ctypes.POINTER(_P)]
    L.fvv_serve_set_frames.argtypes = [_P, ctypes.c_int64, ctypes.c_int, _P]
    L.fvv_serve_submit.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_uint64)]
    L.fvv_serve_poll.argtypes = [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double)]
    L.fvv_serve_release.argtypes = [_P, ctypes.c_uint64]
    L.fvv_serve_stats_get.argtypes = [_P, ctypes.POINTER(fvv_serve_stats)]
    L.fvv_serve_destroy.argtypes = [_P]
    L.fvv_serve_calibrate_fp8.argtypes = [_P, ctypes.c_int, _P, ctypes.c_int]
    L._serve_ready = True
    return L


def fvv_serve_default_cfg(**kw) -> fvv_serve_cfg:
    c = fvv_serve_cfg()
    _serve_sigs(lib()).fvv_serve_default_cfg(ctypes.byref(c))
    for k, v in kw.items():
        if k in ("res_h", "res_w"):
            for i, x in enumerate(v):
                getattr(c, k)[i] = int(x)
        else:
            setattr(c, k, v)
    return c


def fvv_serve_create(weights, cfg: fvv_serve_cfg) -> int:
    L = _serve_sigs(lib())
    if weights is None:
        wp, n = None, 0
    else:
        w, wp = _host_f32(weights)
        n = w.size
    s = _P()
    _check(L.fvv_serve_create(wp, n, ctypes.byref(cfg), ctypes.byref(s)))
    return s.value


def fvv_serve_calibrate_fp8(s: int, res_id: int, frames, n_pairs: int):
    """FP8 server: activation scales of every slot of one resolution (see fvv.h)."""
    _check(_serve_sigs(lib()).fvv_serve_calibrate_fp8(s, res_id, _dev(frames), n_pairs))


def fvv_serve_set_frames(s: int, instant: int, res_id: int, cams):
    ptrs = (ctypes.c_void_p * len(cams))(*[_dev(c) for c in cams])
    _check(_serve_sigs(lib()).fvv_serve_set_frames(s, instant, res_id, ptrs))


def fvv_serve_submit(s: int, user: int, pair: int, t: float, res_id: int) -> int:
    tk = ctypes.c_uint64()
    _check(_serve_sigs(lib()).fvv_serve_submit(s, user, pair, float(t), res_id, ctypes.byref(tk)))
    return tk.value


def fvv_serve_poll(s: int, ticket: int):
    """(state, device pointer, latency_ms): state 0 done, 1 pending; raises on errors."""
    p, lat = ctypes.c_void_p(), ctypes.c_double()
    rc = _serve_sigs(lib()).fvv_serve_poll(s, ticket, ctypes.byref(p), ctypes.byref(lat))
    if rc < 0:
        raise FvvError(rc, lib().fvv_last_error().decode())
    return rc, p.value, lat.value


def fvv_serve_release(s: int, ticket: int) -> int:
    rc = _serve_sigs(lib()).fvv_serve_release(s, ticket)
    if rc < 0:
        raise FvvError(rc, lib().fvv_last_error().decode())
    return rc


def fvv_serve_stats_get(s: int) -> dict:
    st = fvv_serve_stats()
    _check(_serve_sigs(lib()).fvv_serve_stats_get(s, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in fvv_serve_stats._fields_}


def fvv_serve_destroy(s: int):
    _serve_sigs(lib()).fvv_serve_destroy(s)


def fvv_calibrate_fp8(h: int, frames, n_pairs: int, stream=None):
    """frames: CUDA float32 tensor n_pairs x 2 x H x W x 3 (left, right of each pair)."""
    L = lib()
    L.fvv_calibrate_fp8.argtypes = [_P, _P, ctypes.c_int, _P]
    _check(L.fvv_calibrate_fp8(h, _dev(frames), n_pairs, _stream(stream)))


def fvv_interp_fp8_scales(h: int, layer: int, n: int):
    """(s_a, s_w[:n]) of an FP8 layer after calibration."""
    L = lib()
    L.fvv_interp_fp8_scales.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_int]
    sa = ctypes.c_float()
    sw = np.zeros(n, np.float32)
    _check(L.fvv_interp_fp8_scales(h, layer, ctypes.byref(sa), sw.ctypes.data, n))
    return sa.value, sw
