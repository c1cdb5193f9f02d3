"""Seeded He-initialised weight blob for the VINet architecture (Table 3).

This module only draws random numbers in a fixed order; it holds none of the
network's arithmetic.  The blob is a flat float32 array, layer by layer in the
manifest order below, each layer as W then b:

* Conv2d 3x3 (pad 1, stride 1 or 2): W laid out [C_out][C_in][3][3]
* ConvTranspose2d 4x4 (stride 2, pad 1): W laid out [C_in][C_out][4][4]

Initialisation (He): W ~ N(0, 2 / fan_in) with fan_in = C_in * 9 for a 3x3 conv
and C_in * 4 for the 4x4 stride-2 transposed conv (each output pixel sees 2x2
taps per input channel); b ~ U(-0.01, 0.01).  Generator: numpy PCG64(seed),
drawing W (standard normal, float64, then scaled) and b in manifest order.

The layer list is restated from Table 3 (VIBlock_i, ContextNet, RefineNet);
channel counts of concatenated inputs follow the context-aware U-Net reading
(RefineNet encoder level k>0 input = [previous, left ctx_k, right ctx_k],
decoders take [previous decoder, mirrored encoder]).
"""
from __future__ import annotations

import numpy as np

CONV, CONVT = "conv", "convT"


def _vib(i: int, c_in: int):
    p = f"vib{i}."
    rows = [(p + "c0", CONV, c_in, 128, 2, True),
            (p + "c1", CONV, 128, 256, 2, True)]
    rows += [(p + f"m{k}", CONV, 256, 256, 1, True) for k in range(6)]
    rows += [(p + "t0", CONVT, 256, 128, 2, True),
             (p + "t1", CONVT, 128, 5, 2, False)]
    return rows


def manifest():
    """(name, kind, C_in, C_out, stride, relu) for every layer, in blob order."""
    rows = _vib(0, 7) + _vib(1, 18) + _vib(2, 18)
    ctx = [(3, 16, 2), (16, 16, 1), (16, 32, 2), (32, 32, 1),
           (32, 64, 2), (64, 64, 1), (64, 128, 2), (128, 128, 1)]
    rows += [(f"ctx.c{k}", CONV, ci, co, s, True) for k, (ci, co, s) in enumerate(ctx)]
    ref = [("e0a", CONV, 6, 32, 2, True), ("e0b", CONV, 32, 32, 1, True),
           ("e1a", CONV, 64, 64, 2, True), ("e1b", CONV, 64, 64, 1, True),
           ("e2a", CONV, 128, 128, 2, True), ("e2b", CONV, 128, 128, 1, True),
           ("e3a", CONV, 256, 256, 2, True), ("e3b", CONV, 256, 256, 1, True),
           ("d0", CONVT, 512, 128, 2, True), ("d1", CONVT, 256, 64, 2, True),
           ("d2", CONVT, 128, 32, 2, True), ("d3", CONVT, 64, 16, 2, True),
           ("out", CONV, 16, 3, 1, False)]
    rows += [("ref." + n, k, ci, co, s, r) for n, k, ci, co, s, r in ref]
    return rows


def layer_sizes(kind: str, c_in: int, c_out: int):
    taps = 9 if kind == CONV else 16
    return c_in * c_out * taps, c_out


def n_floats() -> int:
    return sum(sum(layer_sizes(k, ci, co)) for _, k, ci, co, _, _ in manifest())


def he_init(seed: int = 0) -> np.ndarray:
    """Flat float32 blob of all weights and biases (see module docstring)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for _, kind, ci, co, _, _ in manifest():
        nw, nb = layer_sizes(kind, ci, co)
        fan_in = ci * (9 if kind == CONV else 4)
        w = rng.standard_normal(nw) * np.sqrt(2.0 / fan_in)
        b = rng.uniform(-0.01, 0.01, nb)
        parts += [w, b]
    return np.concatenate(parts).astype(np.float32)


def layer_views(blob: np.ndarray):
    """Dict name -> (W array in its PyTorch layout, b) viewing the blob."""
    out, off = {}, 0
    for name, kind, ci, co, _, _ in manifest():
        nw, nb = layer_sizes(kind, ci, co)
        shape = (co, ci, 3, 3) if kind == CONV else (ci, co, 4, 4)
        out[name] = (blob[off:off + nw].reshape(shape), blob[off + nw:off + nw + nb])
        off += nw + nb
    assert off == blob.size
    return out
