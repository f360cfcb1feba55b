"""Seeded synthetic patch layouts on the unit sphere.

These generators produce the inputs (patch centres, radii, modes) that both the
CUDA path and the CPU oracle consume. They contain none of the solver's
arithmetic: only random sampling, the Fibonacci spiral and a separation filter.

Workload recipes (Kaye & Greengard, Section 9):
  * area fraction f = N sin^2(eps/2) ~ eps^2 N / 4, so eps = 2 sqrt(f/N)
    (Section 9, eq. patareafrac);
  * patches must be well separated: geodesic centre distance >= 3 eps
    (Section 3);
  * Example 2 places centres on a Fibonacci spiral; Example 3 uses 20
    clusters centred at the vertices of a dodecahedron.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 1906042090


def rng(config_index: int = 0, extra: int = 0) -> np.random.Generator:
    """PCG64 generator seeded from the project base seed."""
    return np.random.Generator(np.random.PCG64([BASE_SEED + config_index, extra]))


def eps_from_area_fraction(f: float, N: int) -> float:
    """Patch radius from area fraction, eps = 2 sqrt(f/N) (Section 9)."""
    return 2.0 * math.sqrt(f / N)


def _chord(geodesic: float) -> float:
    return 2.0 * math.sin(0.5 * geodesic)


class _CellHash:
    """Uniform 3-D cell hash used to enforce a minimum chord distance."""

    def __init__(self, min_chord: float):
        self.h = max(min_chord, 1e-12)
        self.min2 = min_chord * min_chord
        self.cells: dict[tuple[int, int, int], list[int]] = {}
        self.pts: list[np.ndarray] = []

    def _key(self, p):
        return (int(math.floor(p[0] / self.h)), int(math.floor(p[1] / self.h)),
                int(math.floor(p[2] / self.h)))

    def ok(self, p) -> bool:
        kx, ky, kz = self._key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for idx in self.cells.get((kx + dx, ky + dy, kz + dz), ()):
                        q = self.pts[idx]
                        d2 = (p[0] - q[0]) ** 2 + (p[1] - q[1]) ** 2 + (p[2] - q[2]) ** 2
                        if d2 < self.min2:
                            return False
        return True

    def add(self, p):
        self.cells.setdefault(self._key(p), []).append(len(self.pts))
        self.pts.append(p)


def uniform(N: int, eps: float, gen: np.random.Generator, sep: float = 3.0,
            max_tries: int = 200_000_000) -> np.ndarray:
    """Uniform centres (normalised Gaussian 3-vectors), rejecting any draw
    within geodesic sep*eps of an accepted centre."""
    H = _CellHash(_chord(sep * eps))
    out = np.empty((N, 3))
    n = 0
    tries = 0
    while n < N:
        batch = gen.standard_normal((4096, 3))
        batch /= np.linalg.norm(batch, axis=1, keepdims=True)
        for p in batch:
            tries += 1
            if H.ok(p):
                H.add(p)
                out[n] = p
                n += 1
                if n == N:
                    break
        if tries > max_tries:
            raise RuntimeError("uniform layout: separation infeasible")
    return out


def fibonacci(N: int) -> np.ndarray:
    """Fibonacci spiral: z_k = 1 - (2k+1)/N, phi_k = k pi (3 - sqrt 5)."""
    k = np.arange(N, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / N
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def _tangent_basis(c):
    a = np.array([0.0, 0.0, 1.0]) if abs(c[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    e1 = np.cross(a, c)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(c, e1)
    return e1, e2


def _move(c, dist, ang):
    e1, e2 = _tangent_basis(c)
    d = math.cos(ang) * e1 + math.sin(ang) * e2
    p = math.cos(dist) * c + math.sin(dist) * d
    return p / np.linalg.norm(p)


def jittered_fibonacci(N: int, eps: float, gen: np.random.Generator, frac: float = 0.3,
                       sep: float = 3.0) -> np.ndarray:
    """Fibonacci spiral with a seeded jitter of frac * sqrt(4 pi / N) in a uniform
    random tangent direction; a point that violates the sep*eps separation
    redraws its jitter (and keeps its spiral position after 64 failed draws)."""
    base = fibonacci(N)
    J = frac * math.sqrt(4.0 * math.pi / N)
    H = _CellHash(_chord(sep * eps))
    out = np.empty_like(base)
    for i in range(N):
        placed = False
        for _ in range(64):
            p = _move(base[i], J * math.sqrt(gen.uniform()), gen.uniform(0, 2 * math.pi))
            if H.ok(p):
                placed = True
                break
        if not placed:
            p = base[i]
            if not H.ok(p):
                raise RuntimeError("jittered Fibonacci: cannot place point %d" % i)
        H.add(p)
        out[i] = p
    return out


def dodecahedron_vertices() -> np.ndarray:
    """The 20 unit vertices of a regular dodecahedron."""
    ph = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                v.append((sx, sy, sz))
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            v.append((0, s1 / ph, s2 * ph))
            v.append((s1 / ph, s2 * ph, 0))
            v.append((s2 * ph, 0, s1 / ph))
    v = np.array(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _vmf_sample(mu, kappa, gen):
    # Wood (1994) sampler for the 3-D von Mises-Fisher distribution.
    u = gen.uniform()
    w = 1.0 + math.log(u + (1.0 - u) * math.exp(-2.0 * kappa)) / kappa
    ang = gen.uniform(0, 2 * math.pi)
    s = math.sqrt(max(0.0, 1.0 - w * w))
    e1, e2 = _tangent_basis(mu)
    p = w * mu + s * (math.cos(ang) * e1 + math.sin(ang) * e2)
    return p / np.linalg.norm(p)


def vmf_clusters(N: int, eps: float, gen: np.random.Generator, kappa: float = 50.0,
                 sep: float = 3.0, max_tries: int = 100_000_000) -> np.ndarray:
    """20 equally weighted von Mises-Fisher clusters with mean directions at the
    dodecahedron vertices; rejection enforces the sep*eps separation."""
    mus = dodecahedron_vertices()
    H = _CellHash(_chord(sep * eps))
    out = np.empty((N, 3))
    n = 0
    tries = 0
    while n < N:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("vMF layout: separation infeasible")
        p = _vmf_sample(mus[gen.integers(20)], kappa, gen)
        if H.ok(p):
            H.add(p)
            out[n] = p
            n += 1
    return out


def min_geodesic_separation(c: np.ndarray) -> float:
    """Smallest geodesic distance between two centres (brute force for small N,
    cell hash otherwise)."""
    N = len(c)
    if N < 2:
        return math.pi
    if N <= 4000:
        g = np.clip(c @ c.T, -1.0, 1.0)
        np.fill_diagonal(g, -2.0)
        return float(np.arccos(g.max()))
    # approximate neighbourhood search on a cell hash of the mean spacing
    h = 4.0 * math.sqrt(4.0 * math.pi / N)
    keys = np.floor(c / h).astype(np.int64)
    cells: dict = {}
    for i, k in enumerate(map(tuple, keys)):
        cells.setdefault(k, []).append(i)
    best = 2.0
    for i, k in enumerate(map(tuple, keys)):
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in cells.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                        if j != i:
                            d = float(np.linalg.norm(c[i] - c[j]))
                            best = min(best, d)
    return 2.0 * math.asin(min(1.0, best / 2.0))


# ---------------------------------------------------------------------------
# The named workloads. Index = position in the workload list:
#   0: exterior, N=10, eps=0.05, K=64, uniform
#   1: interior, N=1000, eps=0.02, K=128, uniform
#   2: exterior, N=10000, eps=0.005, K=136, jittered Fibonacci
#   3: N=100000, eps=0.001, K=136, jittered Fibonacci or 20 vMF clusters
#   4: 256 independent spheres (batched)
# ---------------------------------------------------------------------------

def workload(index: int, layout: str = "fibonacci", N: int | None = None):
    """Return (centres, eps, mode, K) for one of the named single-sphere workloads.
    mode: 0 = exterior (narrow capture), 1 = interior (narrow escape)."""
    g = rng(index)
    if index == 0:
        n = N or 10
        return uniform(n, 0.05, g), 0.05, 0, 64
    if index == 1:
        n = N or 1000
        return uniform(n, 0.02, g), 0.02, 1, 128
    if index == 2:
        n = N or 10000
        return jittered_fibonacci(n, 0.005, g), 0.005, 0, 136
    if index == 3:
        n = N or 100000
        if layout == "fibonacci":
            return jittered_fibonacci(n, 0.001, g), 0.001, 1, 136
        return vmf_clusters(n, 0.001, g), 0.001, 1, 136
    raise ValueError(index)


def batch_workload(B: int = 256, seed_index: int = 4):
    """Batch of independent spheres: N_b log-uniform in [50, 5000], eps_b uniform in
    [0.005, min(0.02, sqrt(0.62/N_b))] (capped so the 3*eps exclusion discs cover at
    most ~35% of the sphere), mode = b mod 2, uniform centres, K = 128."""
    g = rng(seed_index)
    out = []
    for b in range(B):
        Nb = int(round(math.exp(g.uniform(math.log(50), math.log(5000)))))
        hi = min(0.02, math.sqrt(0.62 / Nb))
        eb = g.uniform(0.005, max(0.005, hi))
        cb = uniform(Nb, eb, rng(seed_index, b + 1))
        out.append((cb, eb, b % 2, 128))
    return out
