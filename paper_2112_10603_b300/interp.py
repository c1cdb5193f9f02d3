"""Interpolator: owns one fvv_interp handle and allocates outputs with torch."""
from __future__ import annotations

import numpy as np

from . import _lib as L


class Interpolator:
    def __init__(self, weights, H: int, W: int, precision: int = L.FVV_FP32, pad_mode: int = L.FVV_PAD_ZERO,
                 max_views: int = 16, max_cams: int = 2, t_mode: int = L.FVV_T_DIRECT, graphs: int = 1):
        self.H, self.W = H, W
        self.opts = L.fvv_default_opts(precision=precision, pad_mode=pad_mode, max_views=max_views,
                                       max_cams=max_cams, t_mode=t_mode, graphs=graphs)
        self.h = L.fvv_interp_create(weights, H, W, self.opts)

    def run(self, left, right, t, out=None, stream=None):
        """left/right: CUDA float32 H x W x 3 tensors; t: sequence of positions."""
        import torch
        t = np.atleast_1d(np.asarray(t, np.float32))
        if out is None:
            out = torch.empty((len(t), self.H, self.W, 3), dtype=torch.float32, device=left.device)
        L.fvv_interp_run(self.h, left, right, t, len(t), out, stream)
        return out

    def run_host(self, left, right, t, out=None):
        t = np.atleast_1d(np.asarray(t, np.float32))
        if out is None:
            out = np.empty((len(t), self.H, self.W, 3), np.float32)
        L.fvv_interp_run_host(self.h, left, right, t, len(t), out, None)
        return out

    def submit_host(self, left, right, t, out):
        """Pipelined host-buffer call: returns a ticket for wait_host.  left, right, out:
        float32 host buffers (pinned tensors for overlap) kept alive until the wait."""
        t = np.atleast_1d(np.asarray(t, np.float32))
        return L.fvv_interp_submit_host(self.h, left, right, t, len(t), out, None)

    def wait_host(self, ticket: int):
        L.fvv_interp_wait_host(self.h, ticket)

    def run_batch(self, cams, pair_left, view_offsets, t, out=None, stream=None):
        import torch
        t = np.asarray(t, np.float32)
        if out is None:
            out = torch.empty((len(t), self.H, self.W, 3), dtype=torch.float32, device=cams[0].device)
        L.fvv_interp_run_batch(self.h, cams, pair_left, view_offsets, t, out, stream)
        return out

    def autotune(self, n_views: int, cache_path: str | None = None):
        """Pick each tensor-core layer's tile rectangle by measurement (JSON cache)."""
        L.fvv_interp_autotune(self.h, n_views, cache_path)

    def peek(self, which: str, view: int = 0):
        """Intermediates of the last run: 'vib0'|'vib1'|'vib2'|'blend'|'z' (padded grid)."""
        Hp, Wp = -(-self.H // 16) * 16, -(-self.W // 16) * 16
        if which.startswith("vib"):
            s = int(which[3])
            f = 2 ** (2 - s)
            return L.fvv_interp_peek(self.h, s, view, (Hp // f, Wp // f, 5))
        return L.fvv_interp_peek(self.h, {"blend": 3, "z": 4}[which], view, (Hp, Wp, 3))

    @property
    def device_bytes(self) -> int:
        return L.fvv_interp_device_bytes(self.h)

    @property
    def last_launches(self) -> int:
        return L.fvv_interp_last_launches(self.h)

    @property
    def graph_captures(self) -> int:
        return L.fvv_interp_graph_captures(self.h)

    def close(self):
        if self.h:
            L.fvv_interp_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
