"""Neumann Green's functions of the unit sphere (Kaye & Greengard, Section 2.1).

Test infrastructure only (see the package docstring).

mode 0 = exterior (narrow capture, G_E), mode 1 = interior (narrow escape, G_I).
"""
import numpy as np

EXTERIOR = 0
INTERIOR = 1


def G_on_surface(d, mode):
    """G for two points on the sphere as a function of their chord distance d.

    Exterior, eq. (Gextonsurface): 2/d - log(2/d) - log(1 + d/2).
    Interior, eq. (Gintonsurface): 2/d + log(2/d) - log(1 + d/2).
    """
    d = np.asarray(d, dtype=np.float64)
    s = -1.0 if mode == EXTERIOR else 1.0
    return 2.0 / d + s * np.log(2.0 / d) - np.log1p(0.5 * d)


def G_off_surface(x, xp, mode):
    """G(x, x') for x' on the unit sphere and x anywhere in the closed domain.

    Exterior, eq. (Gextoffsurface): 2/|x-x'| + log((|x| - x.x') / (1 - x.x' + |x-x'|)).
    Interior, eq. (Gintoffsurface): 2/|x-x'| + log(2 / (1 - x.x' + |x-x'|)).
    x, xp: arrays (..., 3).
    """
    x = np.asarray(x, dtype=np.float64)
    xp = np.asarray(xp, dtype=np.float64)
    diff = x - xp
    d = np.sqrt(np.sum(diff * diff, axis=-1))
    xx = np.sum(x * xp, axis=-1)
    if mode == EXTERIOR:
        rx = np.sqrt(np.sum(x * x, axis=-1))
        return 2.0 / d + np.log((rx - xx) / (1.0 - xx + d))
    return 2.0 / d + np.log(2.0 / (1.0 - xx + d))


def chord(x, xp):
    """|x - x'| for arrays of 3-vectors (broadcasting)."""
    diff = np.asarray(x, dtype=np.float64) - np.asarray(xp, dtype=np.float64)
    return np.sqrt(np.sum(diff * diff, axis=-1))
