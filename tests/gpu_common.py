"""Shared fixtures of the GPU parity tests: seeded inputs and cached oracle runs."""
import functools

import numpy as np

import oracle
from synth import scene, weights


@functools.lru_cache(maxsize=None)
def blob(seed: int = 0):
    return weights.he_init(seed)


@functools.lru_cache(maxsize=None)
def pair(seed: int, H: int, W: int, max_disp: float):
    return scene.stereo_pair(seed, H, W, max_disp)


@functools.lru_cache(maxsize=None)
def oracle_view(seed: int, H: int, W: int, max_disp: float, t: float, circ: bool = False):
    left, right = pair(seed, H, W, max_disp)
    return oracle.vinet_forward(blob(), left, right, t, circ=circ, dumps=True)


def psnr(a, b):
    mse = np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2)
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)
