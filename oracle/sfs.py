"""Shape-from-shading forcing (CPU reference).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Passage followed: the shape-from-shading section, Eq. (SfS-forcingFunc).  A
Lambertian surface lit from the vertical direction images as
P = 1 / sqrt(|grad S*|^2 + 1); the height field S* solves the eikonal
equation with f = sqrt(1 / P^2 - 1), seeded with known heights.  Reading
used here and by the CUDA path: P must lie in (0, 1]; f is raised to f_min
where the formula gives less (flat image regions, P = 1, would give f = 0,
which the solver does not accept); P outside (0, 1] or not finite gives NaN.
"""
from __future__ import annotations

import numpy as np


def forcing(P: np.ndarray, f_min: float) -> np.ndarray:
    P = np.asarray(P, dtype=np.float64)
    out = np.full(P.shape, np.nan)
    ok = np.isfinite(P) & (P > 0.0) & (P <= 1.0)
    f = np.sqrt(1.0 / (P[ok] * P[ok]) - 1.0)
    out[ok] = np.maximum(f, f_min)
    return out


def image_of_height(grad_sq: np.ndarray) -> np.ndarray:
    """Forward imaging operator: P = 1 / sqrt(|grad S*|^2 + 1)."""
    return 1.0 / np.sqrt(np.asarray(grad_sq, dtype=np.float64) + 1.0)
