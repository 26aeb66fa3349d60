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


def test_off_resonance_enters_like_a_gradient_field(oracle_mod):
    """A field deviation ΔB0 along z must turn a spin exactly as a gradient field of the same size
    does: a spin at the centre with Δω = dw_from_b0(G·x0) and no gradient gives the signal of a
    spin at x0 in the gradient G (Eqs. 3.11, 3.13: both are fields along z in the rotating frame).
    The opposite sign would give the complex conjugate phase history and fails."""
    g, x0 = 3e-3, 0.07  # 3 mT/m, 7 cm
    rows = [(0.0, 0.0, 0.0, 0.0, math.pi / 2, 0.3, 0, 0.0)]
    for k in range(40):
        rows.append((25e-6, g, 0.0, 0.0, 0.0, 0.0, 1, 0.0))
        if k == 19:
            rows.append((0.0, 0.0, 0.0, 0.0, 2.0, 1.1, 0, 0.0))
    grad = W.Sequence(W.make_events(rows), W.GAMMA_BAR)
    ev = grad.events.copy()
    ev["gx"] = 0.0
    nograd = W.Sequence(ev, W.GAMMA_BAR)
    one = lambda x, dw: W.Phantom(*(np.array([v], dtype=float) for v in (x, 0.0, 0.0, 1.0, 0.8, 0.05, dw)))
    s_grad = oracle_mod.signal(one(x0, 0.0), grad)
    s_b0 = oracle_mod.signal(one(0.0, float(W.dw_from_b0(g * x0))), nograd)
    assert np.max(np.abs(s_grad - s_b0)) < 1e-12
    assert np.max(np.abs(s_grad - s_grad.conj())) > 0.1  # the phases are not trivially symmetric
    assert W.dw_from_b0(1e-6) == pytest.approx(2 * math.pi * W.GAMMA_BAR * 1e-6, rel=1e-15)


def test_legendre_workload(oracle_mod):
    """The C2 variant with the Eq. 6.3 field: Δω of every water spin is +γΔB0 of its position, fat
    spins add the chemical shift; spins at the centre of the homogeneity sphere see no field."""
    w = W.config2_legendre(n=32, iso=2)
    ph = w.phantom
    b0 = W.b0_legendre(ph.x, ph.y, ph.z, 20e-6, 0.25)
    water = np.tile([True, False], ph.n // 2)
    assert np.allclose(ph.dw[water], 2 * math.pi * W.GAMMA_BAR * b0[water], rtol=1e-14, atol=0)
    assert np.allclose(ph.dw[~water] - 2 * math.pi * W.GAMMA_BAR * b0[~water], 2 * math.pi * W.FAT_SHIFT_HZ,
                       rtol=1e-12, atol=1e-9)
    assert np.max(np.abs(b0)) > 1e-6  # the corners of the 0.5 m field of view leave the sphere


def test_concomitant_components_satisfy_maxwell():
    """The transverse completion of an ideal z-gradient field is divergence- and curl-free: the
    field's Jacobian (rows gtx, gty, G) is traceless and symmetric."""
    rng = np.random.default_rng(5)
    ev = W.make_events([(1e-3, *rng.normal(size=3), 0.0, 0.0, 0, 0.0) for _ in range(20)])
    gt = W.concomitant_transverse(ev)
    for e, g in zip(ev, gt):
        J = np.array([g[:3], g[3:], [e["gx"], e["gy"], e["gz"]]])
        assert abs(np.trace(J)) < 1e-15
        assert np.allclose(J, J.T, atol=0)


def test_field_workload_directions():
    w = W.config_fields()
    assert w.b0_dir.shape == (w.phantom.n, 3)
    assert np.allclose(np.linalg.norm(w.b0_dir, axis=1), 1.0, atol=1e-15)
    tilt = np.arccos(np.clip(w.b0_dir[:, 2], -1, 1))
    assert tilt.max() <= math.radians(10.0) + 1e-12 and tilt.max() > math.radians(5.0)
    assert w.g_transverse.shape == (w.sequence.n_events, 6)
