"""Pins of the oracle's non-parallel-field simulation (§3.2: a static field whose direction differs
from z at a spin; §3.4.3.2: gradient fields with components transverse to z).

The model: the total field at a spin is u = B0*n + b with b = (gtx.x, gty.x, G.x); the spin turns
clockwise about u/|u| by (gamma*(|u| - B0) + dw)*dt (Eqs. 3.5/3.14 in the frame turned to the
field), T2 acts across the field, T1 pulls the component along it towards M0, and every spin
starts at M0*n.  The pins state the same physics independently:

* the Bloch ODE dM/dt = gamma*M x B_eff + relaxation with B_eff along u and the relaxation
  matrix turned to u, integrated exactly by a matrix exponential per event;
* the parallel case (n = z, no transverse components) is the pinned standard oracle;
* a rotation of the whole set-up about z (positions, field directions, gradient vectors and
  their transverse components, RF and receiver phases) leaves the signal unchanged;
* equilibrium along a tilted field is stationary and gives the constant signal M0*(nx + j ny).

A planted-mistake test checks that these pins catch plausible errors in the C code.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from paper_1305_6861_gb300 import workloads as W
from pins import _rf_generator

GAMMA = 2 * math.pi * W.GAMMA_BAR


def unit_vectors(rng, n, max_tilt=math.pi):
    """Directions with polar angle up to max_tilt from z, uniform azimuth."""
    ct = rng.uniform(math.cos(max_tilt), 1.0, n)
    st = np.sqrt(1 - ct**2)
    ph = rng.uniform(0, 2 * math.pi, n)
    return np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)


def field_case(rng, n_spins=5, n_events=60, transverse=True):
    ph = W.random_phantom(n_spins, rng)
    ph.dw[:] = 2 * math.pi * rng.uniform(-80, 80, n_spins)
    ph.t1[:] = rng.uniform(0.05, 2.0, n_spins)
    ph.t2[:] = rng.uniform(0.01, 0.2, n_spins)
    rows = []
    for i in range(n_events):
        flip = rng.uniform(-math.pi, math.pi) if rng.uniform() < 0.2 else 0.0
        g = rng.uniform(-4e-3, 4e-3, 3) if rng.uniform() < 0.7 else np.zeros(3)
        rows.append((rng.uniform(0.0, 2e-4), *g, flip, rng.uniform(0, 2 * math.pi), int(rng.uniform() < 0.5),
                     rng.uniform(0, 2 * math.pi)))
    ev = W.make_events(rows)
    gt = rng.uniform(-3e-3, 3e-3, (n_events, 6)) if transverse else None
    if gt is not None:
        gt[rng.uniform(size=n_events) < 0.3] = 0.0
    return ph, ev, unit_vectors(rng, n_spins), gt


def bruteforce_fields(ph, ev, ndir, gt, b0):
    """Exact solution of the Bloch ODE per event with the field along the total field direction."""
    n_adc = int(np.count_nonzero(ev["adc"]))
    sig = np.zeros(n_adc, dtype=complex)
    for s in range(ph.n):
        x = np.array([ph.x[s], ph.y[s], ph.z[s]])
        n = ndir[s]
        v = np.concatenate([ph.rho[s] * n, [1.0]])
        r1 = 1.0 / ph.t1[s] if np.isfinite(ph.t1[s]) else 0.0
        r2 = 1.0 / ph.t2[s] if np.isfinite(ph.t2[s]) else 0.0
        j = 0
        for i, e in enumerate(ev):
            if e["rf_flip"] != 0.0:
                v = expm(e["rf_flip"] * _rf_generator(e["rf_phase"])) @ v
            b = np.array([0.0, 0.0, e["gx"] * x[0] + e["gy"] * x[1] + e["gz"] * x[2]])
            if gt is not None:
                b[0] = gt[i, :3] @ x
                b[1] = gt[i, 3:] @ x
            u = b0 * n + b
            h = u / np.linalg.norm(u)
            beff = (np.linalg.norm(u) - b0 + ph.dw[s] / GAMMA) * h
            bx = np.array([[0, -beff[2], beff[1]], [beff[2], 0, -beff[0]], [-beff[1], beff[0], 0]])
            A = np.zeros((4, 4))
            A[:3, :3] = -GAMMA * bx - r2 * (np.eye(3) - np.outer(h, h)) - r1 * np.outer(h, h)
            A[:3, 3] = ph.rho[s] * r1 * h
            v = expm(e["dt"] * A) @ v
            if e["adc"]:
                sig[j] += (v[0] + 1j * v[1]) * np.exp(-1j * e["adc_phase"])
                j += 1
    return sig


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def pin_fields_bruteforce(simf):
    rng = np.random.default_rng(61)
    for b0, transverse in ((0.02, True), (0.3, True), (1.5, False), (0.05, False)):
        ph, ev, nd, gt = field_case(rng, transverse=transverse)
        got, _ = simf(ph, ev, W.GAMMA_BAR, nd, gt, b0)
        ref = bruteforce_fields(ph, ev, nd, gt, b0)
        assert rel(got, ref) <= 1e-9, (b0, transverse, rel(got, ref))


def pin_fields_parallel_case(simf, sim):
    rng = np.random.default_rng(62)
    ph, ev, _, _ = field_case(rng, n_spins=40, n_events=300, transverse=False)
    nd = np.tile([0.0, 0.0, 1.0], (ph.n, 1))
    for gt in (None, np.zeros((len(ev), 6))):
        got, st = simf(ph, ev, W.GAMMA_BAR, nd, gt, 1.5, want_state=True)
        ref, rst = sim(ph, ev, W.GAMMA_BAR, want_state=True)
        assert rel(got, ref) <= 1e-12
        assert np.max(np.abs(st - rst)) <= 1e-12


def _rotz(phi):
    c, s = math.cos(phi), math.sin(phi)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def pin_fields_rotation_about_z(simf):
    rng = np.random.default_rng(63)
    ph, ev, nd, gt = field_case(rng, n_spins=30, n_events=120)
    ref, _ = simf(ph, ev, W.GAMMA_BAR, nd, gt, 0.1)
    phi = 0.83
    R = _rotz(phi)
    pos = np.stack([ph.x, ph.y, ph.z], axis=1) @ R.T
    ph2 = W.Phantom(pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy(), ph.rho, ph.t1, ph.t2, ph.dw)
    ev2 = ev.copy()
    g = np.stack([ev["gx"], ev["gy"], ev["gz"]], axis=1) @ R.T
    ev2["gx"], ev2["gy"], ev2["gz"] = g[:, 0], g[:, 1], g[:, 2]
    ev2["rf_phase"] = ev["rf_phase"] + phi
    ev2["adc_phase"] = ev["adc_phase"] + phi
    c, s = math.cos(phi), math.sin(phi)
    gx2 = (c * gt[:, :3] - s * gt[:, 3:]) @ R.T  # the transverse field turns with the frame
    gy2 = (s * gt[:, :3] + c * gt[:, 3:]) @ R.T
    got, _ = simf(ph2, ev2, W.GAMMA_BAR, nd @ R.T, np.concatenate([gx2, gy2], axis=1), 0.1)
    assert rel(got, ref) <= 1e-11


def pin_fields_tilted_equilibrium(simf):
    rng = np.random.default_rng(64)
    ph = W.random_phantom(7, rng)
    nd = unit_vectors(rng, 7, max_tilt=1.2)
    rows = [(rng.uniform(0, 1e-2), 0.0, 0.0, 0.0, 0.0, 0.0, 1, a) for a in rng.uniform(0, 2 * math.pi, 20)]
    ev = W.make_events(rows)
    got, st = simf(ph, ev, W.GAMMA_BAR, nd, None, 1.5, want_state=True)
    m0 = np.sum(ph.rho * (nd[:, 0] + 1j * nd[:, 1]))
    assert np.allclose(got, m0 * np.exp(-1j * ev["adc_phase"]), rtol=0, atol=1e-14)
    assert np.allclose(st, ph.rho[:, None] * nd, rtol=0, atol=1e-14)


FIELD_PINS = [pin_fields_bruteforce, pin_fields_rotation_about_z, pin_fields_tilted_equilibrium]


def _simf(oracle_mod, lib=None):
    def simf(ph, ev, gamma, nd, gt, b0, want_state=False):
        return oracle_mod.simulate_fields(ph, ev, gamma, nd, gt, b0, want_state=want_state, lib=lib)
    return simf


@pytest.mark.parametrize("pin", FIELD_PINS, ids=[p.__name__ for p in FIELD_PINS])
def test_fields_oracle_pin(pin, oracle_mod):
    pin(_simf(oracle_mod))


def test_fields_oracle_reduces_to_the_parallel_oracle(oracle_mod):
    pin_fields_parallel_case(_simf(oracle_mod), oracle_mod.simulate)


def test_fields_oracle_rejects_bad_inputs(oracle_mod):
    ph, ev, nd, gt = field_case(np.random.default_rng(65))
    with pytest.raises(RuntimeError):
        oracle_mod.simulate_fields(ph, ev, W.GAMMA_BAR, nd, gt, 0.0)


FIELD_MUTATIONS = [
    ("turn sense about the field reversed", "M[i] = e2 * (c * p[i] - s * hxp[i])", "M[i] = e2 * (c * p[i] + s * hxp[i])"),
    ("T1 recovers along z", "M[i] = e2 * (c * p[i] - s * hxp[i]) + along * h[i];",
     "M[i] = e2 * (c * p[i] - s * hxp[i]) + (i == 2 ? along : 0.0);"),
    ("transverse gradient x/y swapped", "b[0] = gt[0] * x + gt[1] * y + gt[2] * z;", "b[0] = gt[3] * x + gt[4] * y + gt[5] * z;"),
    ("field excess without the main-field term", "(2.0 * b0 * nb + bb) / (un + b0)", "b[2]"),
    ("start along z", "double M[3] = {rho[s] * n[0], rho[s] * n[1], rho[s] * n[2]};", "double M[3] = {0.0, 0.0, rho[s]};"),
    ("cross product transposed", "h[1] * p[2] - h[2] * p[1]", "h[2] * p[1] - h[1] * p[2]"),
    ("T2 along the field", "M[i] = e2 * (c * p[i] - s * hxp[i]) + along * h[i];",
     "M[i] = (c * p[i] - s * hxp[i]) + e2 * along * h[i];"),
]


@pytest.mark.parametrize("name,old,new", FIELD_MUTATIONS, ids=[m[0] for m in FIELD_MUTATIONS])
def test_field_pins_catch_planted_mistake(name, old, new, oracle_mod, tmp_path):
    src = oracle_mod.source()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    variant = oracle_mod.Variant(src.replace(old, new), str(tmp_path))
    simf = _simf(oracle_mod, variant.lib)
    caught = []
    for pin in FIELD_PINS:
        try:
            pin(simf)
        except AssertionError:
            caught.append(pin.__name__)
    try:
        pin_fields_parallel_case(simf, variant.simulate)
    except AssertionError:
        caught.append("parallel")
    assert caught, f"no pin caught the planted mistake: {name}"
