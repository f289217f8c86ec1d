"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds no arithmetic of the transform: it only draws images.  The
paper names no dataset and its image sizes are lost with its plots, so these
stand in for its workloads:

* gradient + noise (float): x[r, c] = 127.5 + 127.5 sin(2 pi (0.75 c / W
  + 0.5 r / H)) + U(-8, 8), not clipped (a smooth photographic-like field with
  sensor-like noise, range about -8 .. 263);
* uniform integers U{0 .. 4095} (12-bit samples) for the reversible 5/3;
* constant and linear-ramp edge cases.

Random numbers come from numpy's counter-based Philox generator, so the
same seed gives the same image on x86 and Arm hosts.
"""
from __future__ import annotations

import numpy as np

SEED_SMALL = 1705      # 512 x 512 single-level case and the small edge cases
SEED_LARGE = 8266      # 8192 x 8192, 5 levels
SEED_PRECISION = 1606  # 16384 x 16384, 6 levels
SEED_BATCH = 2017      # batched mixed-size workload
SEED_SERVE = 2026      # serving workload


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def gradient_noise(h: int, w: int, seed: int, dtype=np.float32) -> np.ndarray:
    """Smooth sinusoidal gradient in 0..255 plus uniform noise in [-8, 8)."""
    rng = _rng(seed)
    r = np.arange(h, dtype=np.float64)[:, None]
    c = np.arange(w, dtype=np.float64)[None, :]
    base = 127.5 + 127.5 * np.sin(2.0 * np.pi * (0.75 * c / w + 0.5 * r / h))
    noise = rng.random((h, w), dtype=np.float64) * 16.0 - 8.0
    return (base + noise).astype(dtype)


def uniform_int(h: int, w: int, seed: int, hi: int = 4095) -> np.ndarray:
    """Uniform integers in [0, hi], int32."""
    return _rng(seed).integers(0, hi + 1, size=(h, w), dtype=np.int32)


def constant(h: int, w: int, value=100.0, dtype=np.float32) -> np.ndarray:
    return np.full((h, w), value, dtype=dtype)


def ramp(h: int, w: int, a: float = 3.0, b: float = 5.0, dtype=np.float32) -> np.ndarray:
    """x[r, c] = a c + b r."""
    r = np.arange(h)[:, None]
    c = np.arange(w)[None, :]
    return (a * c + b * r).astype(dtype)


def image(wavelet: str, h: int, w: int, seed: int) -> np.ndarray:
    """The standard input of a wavelet: ints for legall53, gradient + noise otherwise."""
    if wavelet == "legall53":
        return uniform_int(h, w, seed)
    return gradient_noise(h, w, seed)
