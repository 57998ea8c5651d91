"""Test-side helpers: golden-file parsing, contour measurements and the oracle's host thread
count (no LB arithmetic)."""
import contextlib
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_constants(name="paper_constants.txt") -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = [s.strip() for s in line.split("=", 1)]
            out[k] = float(Fraction(v)) if "/" in v else float(v)
    return out


def bilinear(phi, x, y):
    ny, nx = phi.shape
    x0, y0 = int(np.floor(x)), int(np.floor(y))
    tx, ty = x - x0, y - y0
    x0 %= nx; y0 %= ny
    x1, y1 = (x0 + 1) % nx, (y0 + 1) % ny
    return ((1 - tx) * (1 - ty) * phi[y0, x0] + tx * (1 - ty) * phi[y0, x1]
            + (1 - tx) * ty * phi[y1, x0] + tx * ty * phi[y1, x1])


def contour_radius(phi, cx, cy, angles, rmax=None, dr=0.05):
    """Distance from (cx, cy) to the first phi = 0 crossing along each ray (linear interp.)."""
    ny, nx = phi.shape
    rmax = rmax or 0.5 * min(nx, ny) - 1
    radii = []
    for th in angles:
        c, s = np.cos(th), np.sin(th)
        prev_r, prev_v = 0.0, bilinear(phi, cx, cy)
        r = dr
        found = np.nan
        while r <= rmax:
            v = bilinear(phi, cx + r * c, cy + r * s)
            if prev_v > 0 >= v:
                found = prev_r + dr * prev_v / (prev_v - v)
                break
            prev_r, prev_v = r, v
            r += dr
        radii.append(found)
    return np.array(radii)


def tip_x(phi, row, cx, direction=+1):
    """phi = 0 crossing along a grid row from column cx in the given direction."""
    line = phi[int(row)]
    i = int(cx)
    while 0 <= i + direction < len(line) and line[i + direction] > 0:
        i += direction
    j = i + direction
    if not (0 <= j < len(line)):
        return np.nan
    return i + direction * line[i] / (line[i] - line[j])


@contextlib.contextmanager
def oracle_threads(n=None):
    """Run the oracle's node loops on n host threads (default: every CPU this process may
    use) inside the block; its results are bit-identical for any count."""
    import oracle
    n = n or len(os.sched_getaffinity(0))
    oracle.set_threads(n)
    try:
        yield n
    finally:
        oracle.set_threads(1)
