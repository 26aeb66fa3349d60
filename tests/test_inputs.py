"""Input generators that carry physics: the Eq. 6.3 static-field inhomogeneity (checked against
Legendre-polynomial facts that do not use the recursion) and its off-resonance (Eqs. 6.1, 6.2)."""
import math

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W


def test_legendre_p12_facts():
    assert W.legendre(12, 1.0) == pytest.approx(1.0, abs=1e-14)
    assert W.legendre(12, 0.0) == pytest.approx(231 / 1024, abs=1e-15)  # (-1)^6 12! / (2^12 (6!)^2)
    x = np.linspace(-1, 1, 101)
    assert np.allclose(W.legendre(12, -x), W.legendre(12, x), atol=1e-14)  # even
    g, wts = np.polynomial.legendre.leggauss(20)  # exact for degree <= 39
    assert np.sum(wts * W.legendre(12, g) ** 2) == pytest.approx(2 / 25, rel=1e-13)
    assert abs(np.sum(wts * W.legendre(12, g) * W.legendre(10, g))) < 1e-14
    assert abs(np.sum(wts * W.legendre(12, g) * g**4)) < 1e-14  # orthogonal to lower degrees


def test_b0_legendre_field():
    c, R = 2e-6, 0.25
    # pole, equator, centre
    assert W.b0_legendre(0, 0, R, c, R) == pytest.approx(-c, rel=1e-14)
    assert W.b0_legendre(R, 0, 0, c, R) == pytest.approx(-c * 231 / 1024, rel=1e-13)
    assert W.b0_legendre(0, 0, 0, c, R) == 0.0
    # (r/R)^12 scaling along a ray and symmetry z -> -z, azimuthal symmetry
    rng = np.random.default_rng(0)
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    b1 = W.b0_legendre(*(0.1 * v), c, R)
    b2 = W.b0_legendre(*(0.2 * v), c, R)
    assert b2 == pytest.approx(b1 * 2**12, rel=1e-12)
    assert W.b0_legendre(v[0], v[1], -v[2], c, R) == pytest.approx(W.b0_legendre(*v, c, R), rel=1e-13)
    phi = 0.7
    rot = (v[0] * math.cos(phi) - v[1] * math.sin(phi), v[0] * math.sin(phi) + v[1] * math.cos(phi), v[2])
    assert W.b0_legendre(*rot, c, R) == pytest.approx(W.b0_legendre(*v, c, R), rel=1e-12)


def test_off_resonance_sign():
    """ω = -γB (Eq. 6.1): a positive field deviation lowers the precession frequency."""
    assert W.dw_from_b0(1e-6) == pytest.approx(-2 * math.pi * W.GAMMA_BAR * 1e-6, rel=1e-15)
