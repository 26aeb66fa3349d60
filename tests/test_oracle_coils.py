"""Pins of the oracle's receive-coil weighting (Eq. 3.25; §6.1 on inhomogeneous receive
sensitivity): each spin's transverse magnetisation is multiplied by its coil's complex
sensitivity before the superposition of a sample.

Pinned against the single-coil oracle (itself pinned in test_oracle_pins.py) through two facts
that do not use the coil code: a homogeneous sensitivity C = 1 is the single-coil signal
(§3.5.2), and the magnetisation is linear in M0 (Eq. 4.1 from thermal equilibrium), so a
sensitivity a + jb gives S(M0·a) + j·S(M0·b) with S the single-coil signal of the phantom whose
M0 is scaled per spin.
"""
import dataclasses

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _scaled(ph, w):
    return dataclasses.replace(ph, rho=ph.rho * w)


def test_homogeneous_sensitivity_is_the_single_coil_signal(oracle_mod):
    w = W.config1()
    ev, g = w.sequence.events, w.sequence.gamma_hz_per_t
    single = oracle_mod.signal(w)
    coils = oracle_mod.simulate_coils(w.phantom, ev, g, np.ones((1, w.phantom.n)))
    assert rel(coils[0], single) <= 1e-14
    # a constant complex factor rotates and scales the whole signal
    c = 0.7 * np.exp(1j * 1.1)
    coils = oracle_mod.simulate_coils(w.phantom, ev, g, np.full((2, w.phantom.n), c))
    assert rel(coils[1], c * single) <= 1e-14


@pytest.mark.parametrize("seed", range(3))
def test_sensitivity_by_linearity_in_m0(oracle_mod, seed):
    rng = np.random.default_rng(700 + seed)
    ph = W.random_phantom(400 + 111 * seed, rng)
    seq = W.random_sequence(500, rng)
    n_coils = 3
    sens = rng.normal(size=(n_coils, ph.n)) + 1j * rng.normal(size=(n_coils, ph.n))
    got = oracle_mod.simulate_coils(ph, seq.events, seq.gamma_hz_per_t, sens)
    for c in range(n_coils):
        re = oracle_mod.signal(_scaled(ph, sens[c].real), seq)
        im = oracle_mod.signal(_scaled(ph, sens[c].imag), seq)
        assert rel(got[c], re + 1j * im) <= 1e-12, c


def test_coil_of_one_spin(oracle_mod):
    """One spin, 90° pulse about x, free precession: s = C·M0·j·exp(−jΔωt)·exp(−t/T2) (§3.5.2)."""
    ph = W.Phantom(np.array([0.0]), np.array([0.0]), np.array([0.0]), np.array([1.0]), np.array([np.inf]),
                   np.array([0.1]), np.array([2 * np.pi * 30.0]))
    dt = 1e-3
    rows = [(0.0, 0, 0, 0, np.pi / 2, 0.0, 0, 0.0)] + [(dt, 0, 0, 0, 0, 0, 1, 0.0)] * 20
    ev = W.make_events(rows)
    t = dt * np.arange(1, 21)
    c = 0.3 - 0.4j
    got = oracle_mod.simulate_coils(ph, ev, W.GAMMA_BAR, np.array([[c]]))[0]
    want = c * 1j * np.exp(-1j * 2 * np.pi * 30.0 * t) * np.exp(-t / 0.1)
    assert np.max(np.abs(got - want)) <= 1e-14


COIL_MUTATIONS = [
    ("conjugated sensitivity", [("sig[2 * j] += cr * wr - ci * wi;", "sig[2 * j] += cr * wr + ci * wi;"),
                                ("sig[2 * j + 1] += cr * wi + ci * wr;", "sig[2 * j + 1] += cr * wi - ci * wr;")]),
    ("spin and coil indices swapped", [("sens[2 * ((size_t)c * (size_t)n_spins + (size_t)s)]",
                                        "sens[2 * ((size_t)s * (size_t)n_coils + (size_t)c)]")]),
    ("weight before demodulation dropped", [("const double wr = M[0] * cph + M[1] * sph, wi = M[1] * cph - M[0] * sph;",
                                             "const double wr = M[0], wi = M[1];")]),
]


@pytest.mark.parametrize("name,edits", COIL_MUTATIONS, ids=[m[0] for m in COIL_MUTATIONS])
def test_coil_pins_catch_planted_mistake(name, edits, oracle_mod, tmp_path):
    bad = oracle_mod.source()
    for old, new in edits:
        assert old in bad, f"mutation anchor not found: {old}"
        bad = bad.replace(old, new)
    variant = oracle_mod.Variant(bad, str(tmp_path))
    rng = np.random.default_rng(703)
    ph = W.random_phantom(300, rng)
    seq = W.random_sequence(400, rng)
    sens = rng.normal(size=(2, ph.n)) + 1j * rng.normal(size=(2, ph.n))
    got = oracle_mod.simulate_coils(ph, seq.events, seq.gamma_hz_per_t, sens, lib=variant.lib)
    ok = True
    for c in range(2):
        re = oracle_mod.signal(_scaled(ph, sens[c].real), seq)
        im = oracle_mod.signal(_scaled(ph, sens[c].imag), seq)
        ok &= rel(got[c], re + 1j * im) <= 1e-12
    assert not ok, f"the linearity pin did not catch: {name}"
