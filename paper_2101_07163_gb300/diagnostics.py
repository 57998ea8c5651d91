"""Crystal-shape diagnostics of an exported phase field (host, numpy), as used to report the
paper's runs: the phi = 0 crossing along a ray (tip positions, Sec. 3.1.2), the arm tips of a
k-fold crystal, the tip speed over a window of samples, and the notch ratio of a six-fold
plate (how far the contour between two arms falls inside the hexagon through their tips).

These read a (ny, nx) array exported by Lattice.field(PHI); nothing here runs on the solver's
path. Positions are in cells, measured from the seed centre (cx, cy) in node coordinates.
"""
from __future__ import annotations

import math

import numpy as np


def _bilinear(phi: np.ndarray, x: float, y: float) -> float:
    i, j = int(x), int(y)
    fx, fy = x - i, y - j
    return ((phi[j, i] * (1 - fx) + phi[j, i + 1] * fx) * (1 - fy)
            + (phi[j + 1, i] * (1 - fx) + phi[j + 1, i + 1] * fx) * fy)


def tip_radius(phi: np.ndarray, cx: float, cy: float, angle_deg: float,
               step: float = 0.25) -> float:
    """Distance from (cx, cy) along the ray at angle_deg (counter-clockwise from +x) to the
    first crossing of phi from > 0 to <= 0, by bilinear interpolation of phi along the ray and
    linear interpolation between the two samples around the crossing. NaN if the ray leaves
    the grid first or starts outside the crystal."""
    ny, nx = phi.shape
    c, s = math.cos(math.radians(angle_deg)), math.sin(math.radians(angle_deg))
    prev_r, prev_v, r = 0.0, None, 0.0
    while True:
        x, y = cx + r * c, cy + r * s
        if x < 0 or y < 0 or x > nx - 2 or y > ny - 2:
            return float("nan")
        v = float(_bilinear(phi, x, y))
        if prev_v is None and v <= 0:
            return float("nan")
        if prev_v is not None and prev_v > 0 >= v:
            return prev_r + (r - prev_r) * prev_v / (prev_v - v)
        prev_r, prev_v, r = r, v, r + step


def arm_tips(phi: np.ndarray, cx: float, cy: float, fold: int = 6,
             offset_deg: float = 0.0) -> list[float]:
    """tip_radius along the fold directions offset_deg + 360 k / fold, k = 0 .. fold-1."""
    return [tip_radius(phi, cx, cy, offset_deg + 360.0 * k / fold) for k in range(fold)]


def orientation_spread(tips: list[float]) -> float:
    """(max - min) / mean of the arm lengths: 0 for a crystal whose arms all grow alike."""
    t = np.asarray(tips, dtype=np.float64)
    return float((t.max() - t.min()) / t.mean())


def notch_ratio(phi: np.ndarray, cx: float, cy: float, offset_deg: float = 0.0) -> float:
    """Six-fold crystals: the mean phi = 0 radius halfway between two arms over the inradius
    of the hexagon through the six tips -- 1 for a faceted hexagon, below 1 as the arms branch
    out, above 1 for a shape rounder than the hexagon."""
    tips = arm_tips(phi, cx, cy, 6, offset_deg)
    mids = arm_tips(phi, cx, cy, 6, offset_deg + 30.0)
    return float(np.mean(mids) / (np.mean(tips) * math.sqrt(3.0) / 2.0))


def tip_speed(times, radii) -> float:
    """Least-squares slope of radius against time (cells per time unit of `times`)."""
    t = np.asarray(times, dtype=np.float64)
    r = np.asarray(radii, dtype=np.float64)
    if t.size < 2:
        raise ValueError("need at least two samples")
    return float(np.polyfit(t, r, 1)[0])


def solid_area(phi: np.ndarray, dx: float = 1.0) -> float:
    """Sum of (1 + phi)/2 dx^2 in FP64 (the solid area of lbmice_stats, on a host array)."""
    return float((0.5 * (1.0 + np.asarray(phi, dtype=np.float64))).sum() * dx * dx)
