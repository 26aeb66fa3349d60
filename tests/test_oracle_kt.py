"""Pins of the K-t oracle (§4.2; oracle/kt.py).

1. Discrete orthogonality (the basis of the K-t / isochromat equivalence, cf. Eq. 5.2): N
   isochromats evenly spread over one cycle of the unit moment Δk and stepped by the spin-based
   oracle (pinned in test_oracle_pins.py) give Σ_s M_xy,s / N = a_0 exactly while every populated
   order stays below N — for random flips, phases, intervals, order shifts of -1..2, flip scale
   B1 and off-resonance.
2. FID: a single pulse gives a_0(t) = j sin(α) e^{jφ} e^{-t/T2} e^{-j2π Δf t} (Eq. 4.2, Eq. 3.5).
3. Spin echo: 90°_x, shift, 180°_y, shift gives a_0 = j e^{-2τ/T2}.
"""
import math

import numpy as np
import pytest

from oracle import kt
from paper_1305_6861_gb300 import workloads as W


def _close(a, b, tol):
    a, b = np.asarray(a), np.asarray(b)
    assert np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b))), float(np.max(np.abs(a - b)))


@pytest.mark.parametrize("seed", range(3))
def test_kt_equals_isochromat_sum(oracle_mod, seed):
    rng = np.random.default_rng(910 + seed)
    n_iso, n_steps = 64, 12
    dk = 5.0  # cycles/m: the unit moment
    t1, t2 = rng.uniform(0.3, 2.0), rng.uniform(0.03, 0.3)
    b1, df = rng.uniform(0.7, 1.3), rng.uniform(-40, 40)
    x = np.arange(n_iso) / (n_iso * dk)
    ph = W.Phantom(x, np.zeros(n_iso), np.zeros(n_iso), np.full(n_iso, 1.0 / n_iso), np.full(n_iso, t1),
                   np.full(n_iso, t2), np.full(n_iso, 2 * math.pi * df))
    rows, ev_rows = [], []
    for k in range(n_steps):
        al, phi = rng.uniform(-math.pi, math.pi), rng.uniform(0, 2 * math.pi)
        tau = rng.uniform(1e-3, 8e-3)
        q = int(rng.integers(-1, 3))
        smp = int(rng.integers(0, 2)) if k < n_steps - 1 else 1
        adc = rng.uniform(0, 2 * math.pi)
        rows.append((al, phi, tau, q, smp, adc))
        ev_rows.append((tau, q * dk / (W.GAMMA_BAR * tau), 0.0, 0.0, b1 * al, phi, smp, adc))
    ref, _ = oracle_mod.simulate(ph, W.make_events(ev_rows), W.GAMMA_BAR)
    got = kt.simulate([t1], [t2], [b1], [df], kt.make_steps(rows), max_order=2 * n_steps + 2)[0]
    _close(got, ref, 1e-12)


def test_kt_fid():
    t2, df, al, phi = 0.05, 17.0, 0.7, 1.2
    rows = [(al, phi, 1e-3, 0, 1, 0.0)] + [(0.0, 0.0, 1e-3, 0, 1, 0.0)] * 30
    got = kt.simulate([1.0], [t2], None, [df], kt.make_steps(rows), max_order=4)[0]
    t = 1e-3 * np.arange(1, 32)
    want = 1j * math.sin(al) * np.exp(1j * phi) * np.exp(-t / t2) * np.exp(-2j * math.pi * df * t)
    _close(got, want, 1e-14)


def test_kt_spin_echo():
    t1, t2, tau = 0.8, 0.07, 6e-3
    rows = [(math.pi / 2, 0.0, tau, 1, 0, 0.0), (math.pi, math.pi / 2, tau, 1, 1, 0.0)]
    got = kt.simulate([t1], [t2], None, None, kt.make_steps(rows), max_order=4)[0]
    _close(got, [1j * math.exp(-2 * tau / t2)], 1e-15)


def test_kt_truncation_drops_high_orders():
    """Populations pushed past ±K are dropped: with K = 1 a stimulated echo that needs order 2 is lost."""
    rows = [(math.pi / 2, 0.0, 1e-3, 1, 0, 0.0), (math.pi / 2, 0.0, 1e-3, 1, 0, 0.0),
            (math.pi / 2, 0.0, 1e-3, -2, 1, 0.0)]
    full = kt.simulate([1.0], [0.1], None, None, kt.make_steps(rows), max_order=4)[0]
    cut = kt.simulate([1.0], [0.1], None, None, kt.make_steps(rows), max_order=1)[0]
    assert abs(full[0]) > 0.1 and abs(full[0] - cut[0]) > 0.05


def test_kt_shift_beyond_all_orders():
    """A shift of more than 2K + 1 orders empties every transverse population (truncation)."""
    rows = [(math.pi / 2, 0.0, 1e-3, 0, 1, 0.0), (0.0, 0.0, 1e-3, 3, 1, 0.0), (0.0, 0.0, 1e-3, -3, 1, 0.0)]
    got = kt.simulate([1.0], [0.1], None, None, kt.make_steps(rows), max_order=0)[0]
    assert abs(got[0]) > 0.9 and got[1] == 0 and got[2] == 0
    full = kt.simulate([1.0], [0.1], None, None, kt.make_steps(rows), max_order=4)[0]
    assert abs(full[2] - got[0] * math.exp(-2e-3 / 0.1)) < 1e-12  # with room the population comes back
