"""The spatial-sampling check of §5.2.3 (mrsim_max_config_k; host only, no GPU needed).

K_max (Eq. 5.1) is pinned on sequences whose configuration paths are worked out by hand, and the
criterion Δx < Δx_max = π / K_max (Eq. 5.2) is checked against its meaning: isochromats spaced
below Δx_max reproduce the K-t result of the oracles exactly, isochromats spaced far above it
alias.
"""
import math

import numpy as np
import pytest

from oracle import kt as ORK
from paper_1305_6861_gb300 import workloads as W

G = W.GAMMA_BAR


def k_of(gx, dt):
    return 2 * math.pi * G * gx * dt


def test_no_pulse_no_configuration(mrsim_lib):
    ev = W.make_events([(1e-3, 5e-3, 0, 0, 0, 0, 1, 0.0)] * 4)
    assert np.all(mrsim_lib.max_config_k(ev, G) == 0.0)
    assert np.all(np.isinf(mrsim_lib.delta_x_max(ev, G)))


def test_moments_before_the_first_pulse_do_not_count(mrsim_lib):
    ev = W.make_events([(1e-3, 9e-3, 0, 0, 0, 0, 0, 0.0), (1e-3, 2e-3, 0, 0, 0.5, 0, 1, 0.0)])
    assert mrsim_lib.max_config_k(ev, G)[0] == pytest.approx(k_of(2e-3, 1e-3), rel=1e-14)


def test_refocusing_adds_segments(mrsim_lib):
    """90° – m – 180° – m: the conjugated configuration reaches 2m (the echo's partner)."""
    g, dt = 3e-3, 2e-3
    ev = W.make_events([(dt, g, 0, 0, math.pi / 2, 0, 0, 0.0), (dt, g, 0, 0, math.pi, 0, 1, 0.0)])
    k = mrsim_lib.max_config_k(ev, G)
    assert k[0] == pytest.approx(2 * k_of(g, dt), rel=1e-14) and k[1] == 0 and k[2] == 0


def test_excursion_inside_a_segment(mrsim_lib):
    """+2m then -m inside one segment: the maximum is the excursion 2m, not the net m."""
    g, dt = 3e-3, 1e-3
    ev = W.make_events([(0.0, 0, 0, 0, 1.0, 0, 0, 0.0), (dt, 2 * g, 0, 0, 0, 0, 0, 0.0), (dt, -g, 0, 0, 0, 0, 1, 0.0)])
    assert mrsim_lib.max_config_k(ev, G)[0] == pytest.approx(k_of(2 * g, dt), rel=1e-14)


def test_axes_are_independent(mrsim_lib):
    ev = W.make_events([(1e-3, 1e-3, -2e-3, 4e-3, 0.3, 0, 1, 0.0), (1e-3, -1e-3, 2e-3, 0, 0.3, 0, 1, 0.0)])
    k = mrsim_lib.max_config_k(ev, G)
    assert k == pytest.approx([2 * k_of(1e-3, 1e-3), 2 * k_of(2e-3, 1e-3), k_of(4e-3, 1e-3)], rel=1e-14)


def test_invalid_events(mrsim_lib):
    ev = W.make_events([(1e-3, np.nan, 0, 0, 0.3, 0, 1, 0.0)])
    with pytest.raises(mrsim_lib.MrsimError):
        mrsim_lib.max_config_k(ev, G)


@pytest.mark.parametrize("n_iso,aliased", [(64, False), (41, False), (8, True)])
def test_criterion_predicts_aliasing(mrsim_lib, oracle_mod, n_iso, aliased):
    """P pulses each followed by one unit of moment (Δk = 5 cycles/m): K_max = 2πPΔk.  N isochromats
    over one cycle (Δx = 1/(NΔk)) match the K-t populations when Δx < Δx_max (N > 2P) and alias
    when N is well below P."""
    rng = np.random.default_rng(2000 + n_iso)
    P, dk, tau = 20, 5.0, 3e-3
    t1, t2 = 1.1, 0.25
    alphas = rng.uniform(0.3, 2.5, P)
    phis = rng.uniform(0, 2 * math.pi, P)
    gx = dk / (G * tau)
    ev = W.make_events([(tau, gx, 0, 0, a, p, 1, 0.0) for a, p in zip(alphas, phis)])
    dx = 1.0 / (n_iso * dk)
    dx_max = mrsim_lib.delta_x_max(ev, G)[0]
    assert dx_max == pytest.approx(1.0 / (2 * P * dk), rel=1e-12)
    assert (dx < dx_max) == (n_iso > 2 * P)
    x = np.arange(n_iso) * dx
    ph = W.Phantom(x, np.zeros(n_iso), np.zeros(n_iso), np.full(n_iso, 1.0 / n_iso), np.full(n_iso, t1),
                   np.full(n_iso, t2), np.zeros(n_iso))
    spins, _ = oracle_mod.simulate(ph, ev, G)
    kt = ORK.simulate([t1], [t2], None, None, ORK.make_steps([(a, p, tau, 1, 1, 0.0) for a, p in zip(alphas, phis)]),
                      max_order=P + 1)[0]
    err = np.max(np.abs(spins - kt))
    if aliased:
        assert err > 1e-3
    else:
        assert err <= 1e-12
