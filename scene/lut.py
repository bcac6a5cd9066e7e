"""256-entry RGBA colour maps (inputs), float32 ``[256][4]``.

A colour map is a lookup table from a normalised scalar to colour and opacity
(Section 2.1).  The tables are inputs; interpolating them is the method's work.
"""
from __future__ import annotations

import numpy as np

from .cubes import SEED_BASE


def linear_lut() -> np.ndarray:
    """L[i] = (t, 1-t, 1/2 + t/2, t) with t = i/255: its alpha channel is the identity."""
    t = (np.arange(256, dtype=np.float64) / 255.0)
    return np.stack([t, 1.0 - t, 0.5 + 0.5 * t, t], axis=1).astype(np.float32)


def ratio_lut() -> np.ndarray:
    """Colour map for line ratios over the domain [0, 1] (same ramp as ``linear_lut``)."""
    return linear_lut()


def perturbed_lut(base: np.ndarray | None = None, sigma: float = 0.05, config_id: int = 5) -> np.ndarray:
    """Target colour map of the differentiation workload: base + N(0, sigma), clamped to [0, 1]."""
    base = linear_lut() if base is None else base
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE + config_id, 31])))
    return np.clip(base + rng.normal(0.0, sigma, size=base.shape), 0.0, 1.0).astype(np.float32)
