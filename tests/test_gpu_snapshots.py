"""Magnetisation snapshots (§7.2: magnetisation data of every spin at chosen times) through the
C-ABI: the state after each chosen event must equal the oracle's final state on that event
prefix, and the signal must be the one without snapshots.  float64: the phase floor of the
stress sequences (as in test_gpu_forward.py); float32: 1e-4 absolute on states of magnitude ≤ 1
(the state tolerance of the float32 resume tests) and 2e-5 on the signal."""
import math

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def phase_floor(ph, ev, gamma):
    g = 2 * math.pi * gamma
    th = (g * (np.abs(ev["gx"]) * np.abs(ph.x).max() + np.abs(ev["gy"]) * np.abs(ph.y).max()
               + np.abs(ev["gz"]) * np.abs(ph.z).max()) + np.abs(ph.dw).max()) * ev["dt"]
    return max(1e-12, 4 * 2.0**-53 * float(np.sqrt(np.sum(th**2))))


@pytest.fixture(scope="module")
def M(mrsim_lib):
    return mrsim_lib


@pytest.fixture(scope="module")
def ctx(M):
    c = M.Context(0)
    yield c
    c.close()


def cases():
    rng = np.random.default_rng(4300)
    w = W.config1()
    ev = w.sequence.events
    yield w.phantom, ev, np.array([0, 66, 67 * 10 + 30, 67 * 40, len(ev) - 1])  # inside readouts too
    for seed in range(2):
        r = np.random.default_rng(4310 + seed)
        ph = W.random_phantom(1200 + 345 * seed, r)
        seq = W.random_sequence(900, r, runs=True)
        snaps = np.sort(r.choice(len(seq.events), size=8, replace=False))
        yield ph, seq.events, snaps


@pytest.mark.parametrize("case", range(3))
def test_snapshots_match_prefix_states(M, ctx, oracle_mod, case):
    ph, ev, snaps = list(cases())[case]
    p = M.Phantom.from_workload_phantom(ctx, ph)
    s_snap = M.Sequence(ctx, ev, W.GAMMA_BAR, snapshots=snaps)
    s_plain = M.Sequence(ctx, ev, W.GAMMA_BAR)
    assert s_snap.n_snapshots == len(snaps)
    ref_sig, _ = oracle_mod.simulate(ph, ev, W.GAMMA_BAR)
    refs = [oracle_mod.simulate(ph, ev[: e + 1], W.GAMMA_BAR, want_signal=False, want_state=True)[1] for e in snaps]
    tol64 = phase_floor(ph, ev, W.GAMMA_BAR)
    for prec in (M.FP64, M.FP32, M.FP32_KAHAN):
        out = np.zeros((len(snaps), ph.n, 3))
        sig = M.simulate(ctx, p, s_snap, prec, snapshots=out)
        plain = M.simulate(ctx, p, s_plain, prec)
        ctx.stream_status()
        if prec == M.FP64:
            # the snapshot program splits merged intervals and the lazy T1 at the snapshots, so the
            # two signals differ by rounding: both stay within the float64 floor of the oracle
            assert rel_l2(sig, plain) <= 2 * tol64
            assert rel_l2(sig, ref_sig) <= tol64
            for q in range(len(snaps)):
                assert np.max(np.abs(out[q] - refs[q])) <= tol64 * max(1.0, np.abs(refs[q]).max()), q
        elif prec == M.FP32_KAHAN:  # compensated: the float64 bars, at least 1e-10
            tolk = max(1e-10, tol64)
            assert rel_l2(sig, ref_sig) <= tolk
            for q in range(len(snaps)):
                assert np.max(np.abs(out[q] - refs[q])) <= tolk * max(1.0, np.abs(refs[q]).max()), q
        else:
            assert rel_l2(sig, ref_sig) <= 2e-5
            for q in range(len(snaps)):
                assert np.max(np.abs(out[q] - refs[q])) <= 1e-4, q


def test_snapshots_device_buffer_and_batch(M, ctx, oracle_mod):
    torch = pytest.importorskip("torch")
    w = W.config1()
    ev = w.sequence.events
    snaps = np.array([100, 2000])
    p = M.Phantom.from_workload_phantom(ctx, w.phantom)
    s = M.Sequence(ctx, ev, W.GAMMA_BAR, snapshots=snaps)
    out = torch.zeros(len(snaps) * w.phantom.n * 3, dtype=torch.float64, device="cuda")
    M.simulate(ctx, p, s, M.FP64, snapshots=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(len(snaps), w.phantom.n, 3)
    for q, e in enumerate(snaps):
        _, st = oracle_mod.simulate(w.phantom, ev[: e + 1], W.GAMMA_BAR, want_signal=False, want_state=True)
        assert np.max(np.abs(got[q] - st)) <= 1e-12
    # a batch ignores snapshots but still steps through them
    sig = torch.zeros(2 * s.n_adc, dtype=torch.float64, device="cuda")
    b = M.Batch(ctx, [p], [s], M.FP64, [sig])
    b.launch()
    torch.cuda.synchronize()
    ref = oracle_mod.signal(w)
    assert rel_l2(sig.cpu().numpy().view(np.complex128), ref) <= 1e-12
    b.close()


def test_snapshots_through_host_compile(M, ctx, oracle_mod):
    """Snapshots compiled by mrsim_compile (no context) and uploaded with mrsim_sequence_create
    give the states of mrsim_sequence_load_snapshots."""
    rng = np.random.default_rng(4400)
    ph = W.random_phantom(700, rng)
    seq = W.random_sequence(600, rng, runs=True)
    snaps = np.sort(rng.choice(len(seq.events), size=5, replace=False))
    p = M.Phantom.from_workload_phantom(ctx, ph)
    comp = M.Compiled(seq.events, W.GAMMA_BAR, snapshots=snaps)
    s1 = M.Sequence.from_compiled(ctx, comp)
    comp.close()
    s2 = M.Sequence(ctx, seq.events, W.GAMMA_BAR, snapshots=snaps)
    assert s1.n_snapshots == s2.n_snapshots == len(snaps)
    tol64 = phase_floor(ph, seq.events, W.GAMMA_BAR)
    a, b = np.zeros((len(snaps), ph.n, 3)), np.zeros((len(snaps), ph.n, 3))
    sa = M.simulate(ctx, p, s1, M.FP64, snapshots=a)
    sb = M.simulate(ctx, p, s2, M.FP64, snapshots=b)
    ctx.stream_status()
    assert np.max(np.abs(a - b)) <= tol64 * max(1.0, np.abs(b).max())
    assert rel_l2(sa, sb) <= tol64
    ref, _ = oracle_mod.simulate(ph, seq.events, W.GAMMA_BAR)
    assert rel_l2(sa, ref) <= tol64
