"""Pins of the oracle's Green's functions and modal kernels against what the paper
and the mathematics fix (Section 2.1, Section 8.1)."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import onepatch
from oracle.kernels import EXTERIOR, INTERIOR, G_off_surface, G_on_surface


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("nmax", [0, 1, 5, 15])
def test_modal_log_closed_form(nmax):
    """The printed closed form for G_n^(2) (Section 8.1) equals brute quadrature."""
    t = np.array([0.01, 0.02, 0.03, 0.05, 0.001, 0.0999])
    tp = np.array([0.02, 0.0199999, 0.01, 0.049, 0.009, 0.0001])
    q = onepatch.modal_log_term(t, tp, nmax)
    c = onepatch.modal_log_closed_form(t, tp, nmax)
    assert np.abs(q - c).max() <= 1e-13 * max(1.0, np.abs(c).max())


@pytest.mark.parametrize("mode,mean", [(INTERIOR, 2.0), (EXTERIOR, 1.0)])
def test_mean_over_sphere(mode, mean):
    """<G_I> = 2 over the sphere (Section 2.3, used for eq. mufromsigma2); <G_E> = 1
    (same computation for the exterior kernel: the unit-sphere capacitance)."""
    v = quad(lambda r: G_on_surface(2 * np.sin(r / 2), mode) * np.sin(r), 0, np.pi, limit=200,
             epsabs=1e-14, epsrel=1e-14)[0] / 2
    assert abs(v - mean) < 1e-12


def test_GI_at_centre():
    """G_I(0, x') = 2 for |x'| = 1 (used in the proof of Section 2.3)."""
    xp = _unit([0.3, -0.4, 0.5])
    assert abs(G_off_surface(np.zeros(3), xp, INTERIOR) - 2.0) < 1e-15


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_on_off_surface_agree(mode):
    """eq. Gextonsurface/Gintonsurface are the restrictions of the off-surface forms."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        x, xp = _unit(rng.standard_normal(3)), _unit(rng.standard_normal(3))
        d = np.linalg.norm(x - xp)
        assert abs(G_off_surface(x, xp, mode) - G_on_surface(d, mode)) < 1e-12 * abs(G_on_surface(d, mode))


@pytest.mark.parametrize("mode,flux", [(INTERIOR, -1.0), (EXTERIOR, 0.0)])
def test_neumann_data(mode, flux):
    """d/dn_x G(x, x') on the sphere away from x' is -1 (interior, eq. Gintproperties with
    symmetry) and 0 (exterior, eq. Gextproperties): radial finite differences."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        xh, xp = _unit(rng.standard_normal(3)), _unit(rng.standard_normal(3))
        h = 1e-5
        if mode == INTERIOR:  # inside the ball, one-sided second-order difference
            f0, f1, f2 = (G_off_surface(r * xh, xp, mode) for r in (1.0, 1 - h, 1 - 2 * h))
            dr = (3 * f0 - 4 * f1 + f2) / (2 * h)
        else:
            f0, f1, f2 = (G_off_surface(r * xh, xp, mode) for r in (1.0, 1 + h, 1 + 2 * h))
            dr = -(3 * f0 - 4 * f1 + f2) / (2 * h)
        assert abs(dr - flux) < 1e-6


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_harmonic_off_surface(mode):
    """The off-surface forms are harmonic in x away from x' (-Laplace G = 4 pi delta)."""
    xp = _unit([0.2, 0.1, 0.9])
    x = (0.6 if mode == INTERIOR else 1.7) * _unit([0.5, -0.3, 0.2])
    h = 1e-3
    lap = -6 * G_off_surface(x, xp, mode)
    for e in np.eye(3):
        lap += G_off_surface(x + h * e, xp, mode) + G_off_surface(x - h * e, xp, mode)
    assert abs(lap / h ** 2) < 1e-5


def test_modal_kernel_matches_2d_integral():
    """G_n(t, t') from the graded theta rule equals scipy adaptive quadrature."""
    for mode in (EXTERIOR, INTERIOR):
        t, tp = 0.03, 0.021
        g = onepatch.modal_kernels(np.array([t]), np.array([tp]), 6, mode)[0]
        for n in (0, 3, 6):
            def f(th):
                d = np.sqrt(4 * np.sin((t - tp) / 2) ** 2 + 4 * np.sin(t) * np.sin(tp) * np.sin(th / 2) ** 2)
                return G_on_surface(d, mode) * np.cos(n * th) / np.pi
            ref = quad(f, 0, np.pi, points=[0.0], limit=400, epsabs=1e-14, epsrel=1e-14)[0]
            assert abs(g[n] - ref) < 1e-11 * max(1.0, abs(ref))
