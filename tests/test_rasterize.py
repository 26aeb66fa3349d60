"""The rasterized stress variant of the event lists (every event cut into pieces of at most 10 µs).

Eq. 4.1 applied to the pieces of one event composes to the step of the whole event: the precession
angles add, E1/E2 over the pieces multiply to those of the whole duration, and the T1 recovery
term ρ(1 − E1) composes with them.  So a rasterized list must give the canonical signal; this pins
the oracle's relaxation and precession (a wrong recovery term or a per-event phase error would
show up as a dependence on the piece count) and the host compiler's merging of pieces back into
the canonical program."""
import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W
from program_interp import interpret


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def test_rasterize_structure():
    rng = np.random.default_rng(3)
    seq = W.random_sequence(300, rng)
    r = W.rasterize(seq, 4e-6)
    ev, rv = seq.events, r.events
    n = np.maximum(1, np.ceil(ev["dt"] / 4e-6 * (1 - 1e-9))).astype(int)
    assert rv.shape[0] == n.sum() and np.all(rv["dt"] <= 4e-6 * (1 + 1e-12))
    start = np.concatenate([[0], np.cumsum(n)[:-1]])
    seg = np.repeat(np.arange(len(ev)), n)
    # duration and gradient moment of every original event are preserved
    assert np.allclose(np.bincount(seg, rv["dt"]), ev["dt"], rtol=1e-13, atol=0)
    for g in ("gx", "gy", "gz"):
        assert np.array_equal(rv[g], np.repeat(ev[g], n))
    # the pulse acts once, at the start; the sample once, at the end
    assert np.array_equal(rv["rf_flip"][start], ev["rf_flip"]) and np.count_nonzero(rv["rf_flip"]) == np.count_nonzero(ev["rf_flip"])
    last = start + n - 1
    assert np.array_equal(rv["adc"][last], ev["adc"]) and rv["adc"].sum() == ev["adc"].sum()
    assert np.array_equal(rv["adc_phase"][last], ev["adc_phase"])
    assert r.n_adc == seq.n_adc


def test_config1_rasterized_event_count():
    """C1 on the 10 µs raster: 1 000 events per 10 ms TR, 64 000 in all."""
    w = W.config1()
    r = W.rasterize(w.sequence)
    assert r.n_events == 64000
    assert int(r.events["adc"].sum()) == 4096


def test_oracle_invariant_under_rasterization(oracle_mod):
    w = W.config1()
    ph = w.phantom
    sub = np.random.default_rng(4).choice(ph.n, 300, replace=False)
    ph = W.Phantom(*(a[sub] for a in ph.arrays()))
    ref = oracle_mod.simulate(ph, w.sequence.events, w.sequence.gamma_hz_per_t)[0]
    r = W.rasterize(w.sequence)
    # float64 floor of an oracle that turns every spin once per event: the cos/sin rounding of
    # each turn changes |M| by up to about 2^-52, i.e. 2·2^-53 per event over 64 000 events
    assert rel_l2(oracle_mod.simulate(ph, r.events, r.gamma_hz_per_t)[0], ref) <= max(1e-12, 2 * 2.0**-53 * r.n_events)


@pytest.mark.parametrize("seed", range(3))
def test_oracle_random_sequences_invariant(oracle_mod, seed):
    rng = np.random.default_rng(40 + seed)
    ph = W.random_phantom(40, rng)
    seq = W.random_sequence(300, rng)
    r = W.rasterize(seq, 4e-6)
    ref, ref_state = oracle_mod.simulate(ph, seq.events, seq.gamma_hz_per_t, want_state=True)
    got, state = oracle_mod.simulate(ph, r.events, r.gamma_hz_per_t, want_state=True)
    # the random lists carry phases of up to ~1e4 rad per event: float64 rounding of the
    # accumulated phase bounds the agreement (each side rounds its own sums)
    assert rel_l2(got, ref) <= 1e-9
    assert np.max(np.abs(state - ref_state)) <= 1e-9


def test_planted_recovery_mistake_depends_on_piece_count():
    """The invariant catches a wrong T1 recovery term: a step Mz ← E1·Mz + ρ(1 + E1) (sign
    slip) applied to one event or to its pieces gives different Mz."""
    t1, rho, dt = 0.8, 1.0, 4e-3

    def wrong(mz, h, n):
        e1 = np.exp(-h / t1)
        for _ in range(n):
            mz = e1 * mz + rho * (1 + e1)
        return mz

    assert abs(wrong(0.2, dt, 1) - wrong(0.2, dt / 4, 4)) > 1e-3


@pytest.mark.parametrize("case", ["c1", "c2", "c3_small"])
def test_rasterized_list_compiles_to_the_canonical_program(case, mrsim_lib):
    """The host compiler merges the pieces back: same operations, same class counts and class
    values within rounding (readout dwells split into pieces become uniform samples again)."""
    M = mrsim_lib
    w = {"c1": W.config1, "c2": W.config2, "c3_small": lambda: W.config3(n=24, iso=1)}[case]()
    seq = w.sequence
    r = W.rasterize(seq)
    a = M.debug_compile(seq.events, seq.gamma_hz_per_t)
    b = M.debug_compile(r.events, r.gamma_hz_per_t)
    assert len(a["ops"]) == len(b["ops"])
    assert np.array_equal(a["ops"]["kind"], b["ops"]["kind"])
    assert np.array_equal(a["ops"]["n"], b["ops"]["n"])
    for k in ("pcls", "e1", "e2", "train", "demod"):
        assert len(a[k]) == len(b[k]), k
        assert np.allclose(a[k], b[k], rtol=1e-12, atol=1e-15), k


@pytest.mark.parametrize("seed", range(3))
def test_rasterized_random_programs_match_oracle(seed, mrsim_lib, oracle_mod):
    """Pieces of split readouts and of mixed-gradient intervals (a head interval flushed before a
    sample that absorbs its constant-gradient tail): the interpreted program against the oracle
    on the same rasterized list."""
    rng = np.random.default_rng(140 + seed)
    ph = W.random_phantom(30, rng)
    seq = W.rasterize(W.random_sequence(300, rng), 4e-6)
    sig, state, _ = interpret(seq.events, seq.gamma_hz_per_t, ph)
    ref, ref_state = oracle_mod.simulate(ph, seq.events, seq.gamma_hz_per_t, want_state=True)
    # as above: the oracle rounds the phase of every piece, the program that of merged intervals
    assert rel_l2(sig, ref) < 1e-9
    assert np.max(np.abs(state - ref_state)) < 1e-9


def test_snapshots_inside_split_intervals(mrsim_lib, oracle_mod):
    """A snapshot after a piece in the middle of a split readout dwell or rest interval ends the
    merge there: the state at the snapshot is the oracle's state on that prefix, and the samples
    are unchanged."""
    rng = np.random.default_rng(77)
    ph = W.random_phantom(40, rng)
    w = W.config1()
    seq = W.rasterize(W.Sequence(w.sequence.events[: 67 * 3], w.sequence.gamma_hz_per_t), 2.5e-6)
    ev = seq.events
    # pieces that are neither the first nor the last of their event: mid-dwell and mid-rest
    mid = np.nonzero((ev["adc"] == 0) & (ev["rf_flip"] == 0))[0]
    snaps = np.sort(rng.choice(mid, size=5, replace=False))
    sig, _, ops, got = interpret(ev, seq.gamma_hz_per_t, ph, snapshots=snaps)
    ref_sig, _ = oracle_mod.simulate(ph, ev, seq.gamma_hz_per_t)
    tol = max(1e-12, 2 * 2.0**-53 * len(ev))
    assert rel_l2(sig, ref_sig) <= tol
    for q, e in enumerate(snaps):
        _, st = oracle_mod.simulate(ph, ev[: e + 1], seq.gamma_hz_per_t, want_signal=False, want_state=True)
        assert np.max(np.abs(got[q] - st)) <= tol, (q, e)
