"""Seeded layout generators: determinism and the 3 eps separation (Section 3)."""
import numpy as np

from paper_1906_04209_gb300 import layouts as L


def test_deterministic_and_separated():
    a = L.uniform(300, 0.02, L.rng(1))
    b = L.uniform(300, 0.02, L.rng(1))
    assert np.array_equal(a, b)
    assert np.allclose(np.linalg.norm(a, axis=1), 1.0)
    assert L.min_geodesic_separation(a) >= 3 * 0.02 * (1 - 1e-12)


def test_fibonacci_and_jitter():
    f = L.fibonacci(1000)
    assert np.allclose(np.linalg.norm(f, axis=1), 1.0)
    assert abs(f[:, 2].mean()) < 1e-12
    j = L.jittered_fibonacci(2000, 0.005, L.rng(2))
    assert L.min_geodesic_separation(j) >= 0.015 * (1 - 1e-12)


def test_vmf_clusters():
    c = L.vmf_clusters(3000, 0.001, L.rng(3))
    assert L.min_geodesic_separation(c) >= 0.003 * (1 - 1e-12)
    mus = L.dodecahedron_vertices()
    assert mus.shape == (20, 3)
    near = np.argmax(c @ mus.T, axis=1)
    counts = np.bincount(near, minlength=20)
    assert counts.min() > 0.5 * counts.mean()


def test_area_fraction():
    assert abs(L.eps_from_area_fraction(0.05, 10) - 0.1414213562373095) < 1e-15
