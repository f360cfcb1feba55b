"""Patch frames: local geodesic polar coordinates about each patch centre.

Test infrastructure only (see the package docstring).

Reading (the paper fixes the polar system only up to the direction of
theta = 0, Section 4): e3 = c, e1 = (z x c)/|z x c| (e1 = x-axis when c is a pole),
e2 = e3 x e1. The local point (t, theta) is
    x = cos t c + sin t (cos theta e1 + sin theta e2),
with t the arclength from the centre (the arc C(t) = (sin t, cos t) of Section 8).
"""
import numpy as np


def frame(c):
    """(e1, e2, e3) for a unit centre c."""
    c = np.asarray(c, dtype=np.float64)
    a = np.array([-c[1], c[0], 0.0])
    na = np.sqrt(a @ a)
    e1 = a / na if na * na >= 1e-24 else np.array([1.0, 0.0, 0.0])
    e2 = np.cross(c, e1)
    return e1, e2, c


def local_to_global(c, t, th):
    """Points (t, theta) of the patch centred at c, as an (n, 3) array."""
    e1, e2, e3 = frame(c)
    t = np.asarray(t, dtype=np.float64)
    th = np.asarray(th, dtype=np.float64)
    st = np.sin(t)
    return (np.cos(t)[:, None] * e3[None, :]
            + (st * np.cos(th))[:, None] * e1[None, :]
            + (st * np.sin(th))[:, None] * e2[None, :])


def patch_points(centres, t, th):
    """(N, n, 3) array of the local points (t, theta) on every patch."""
    return np.stack([local_to_global(c, t, th) for c in centres])


def geodesic(a, b):
    """Great-circle distance between unit vectors."""
    return float(np.arctan2(np.linalg.norm(np.cross(a, b)), np.dot(a, b)))
