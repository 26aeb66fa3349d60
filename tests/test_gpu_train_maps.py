"""Train maps on the GPU: a shaped pulse that recurs with the same sub-pulse flips, precession class
and T1 class (Eq. 3.23, the same pulse in every TR) runs, for each spin, as one affine map of its
state composed at set-up.  The composition is exact algebra (Eq. 4.1 applied to a sequence of
affine steps), so the signal with maps must equal the oracle's at the usual bars (float64: the
phase floor of the sequence, at least 1e-12; float32 2e-5; compensated 1e-10) and the signal
without maps at the same bars; the program's map kinds and the out-of-memory path of their
allocation are checked too."""
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


def n_map_kinds(M, seq):
    ops = M.debug_compile(seq.events, seq.gamma_hz_per_t)["ops"]
    sel = (ops["kind"] == M.OP_RF_TRAIN) & ((ops["flags"] & M.F_TMAP) != 0)
    return len({int(t) for t in ops["tab"][sel]})


def cases():
    """Spin echoes with sinc pulses of 24 and 64 sub-pulses over 8-16 TRs, off-resonance up to
    ±150 Hz, long T2; a spin count with a ragged last block."""
    rng = np.random.default_rng(5100)
    ph = W.random_phantom(3001, rng)
    ph.dw[:] = 2 * math.pi * rng.uniform(-150, 150, ph.n)
    ph.t2[:] = rng.uniform(0.05, 1.5, ph.n)
    yield ph, W.spin_echo(16, 8, 0.5, 12e-3, 30e-3, 10e-6, n_rf=24)
    ph2 = W.random_phantom(1000, rng)
    ph2.dw[:] = 2 * math.pi * rng.uniform(-60, 60, ph2.n)
    yield ph2, W.spin_echo(8, 16, 0.3, 15e-3, 40e-3, 10e-6, n_rf=64)


@pytest.mark.parametrize("case", range(2))
def test_train_maps_match_oracle_and_steps(M, ctx, oracle_mod, case):
    ph, seq = list(cases())[case]
    assert n_map_kinds(M, seq) >= 1  # the shaped pulses recur: the program has map kinds
    ref = oracle_mod.signal(ph, seq)
    p = M.Phantom.from_workload_phantom(ctx, ph)
    s = M.Sequence.from_workload_sequence(ctx, seq)
    floor = phase_floor(ph, seq.events, seq.gamma_hz_per_t)
    bars = {M.FP64: floor, M.FP32: 2e-5, M.FP32_KAHAN: max(1e-10, floor)}
    try:
        for prec, bar in bars.items():
            ctx.set_train_maps(True)
            with_maps = M.simulate(ctx, p, s, prec)
            ctx.set_train_maps(False)
            steps = M.simulate(ctx, p, s, prec)
            ctx.stream_status()
            assert rel_l2(with_maps, ref) <= bar, (prec, rel_l2(with_maps, ref))
            assert rel_l2(with_maps, steps) <= 2 * bar, (prec, rel_l2(with_maps, steps))
    finally:
        ctx.set_train_maps(True)


def test_train_maps_batch_and_state_out(M, ctx, oracle_mod):
    """The batch builds every phantom's maps in its own launch (and again in a graph replay); the
    final states of a single launch with maps equal the oracle's."""
    torch = pytest.importorskip("torch")
    pairs = list(cases())
    refs = [oracle_mod.signal(ph, seq) for ph, seq in pairs]
    phs = [M.Phantom.from_workload_phantom(ctx, ph) for ph, _ in pairs]
    sqs = [M.Sequence.from_workload_sequence(ctx, seq) for _, seq in pairs]
    outs = [torch.zeros(2 * q.n_adc, dtype=torch.float64, device="cuda") for q in sqs]
    b = M.Batch(ctx, phs, sqs, M.FP32, outs)
    for graph in (False, True, True):
        b.launch(graph=graph)
        torch.cuda.synchronize()
        ctx.stream_status()
        for o, r in zip(outs, refs):
            assert rel_l2(o.cpu().numpy().view(np.complex128), r) <= 2e-5
    b.close()
    ph, seq = pairs[1]
    _, ref_state = oracle_mod.simulate(ph, seq.events, seq.gamma_hz_per_t, want_signal=False, want_state=True)
    state = np.zeros((ph.n, 3))
    M.simulate(ctx, phs[1], sqs[1], M.FP64, state_out=state)
    assert np.max(np.abs(state - ref_state)) <= 1e-12 * max(1.0, np.abs(ref_state).max())


def test_train_map_allocation_failure(M, ctx, oracle_mod):
    """The maps' device memory (the context's stream-ordered pool) failing gives MRSIM_ENOMEM and
    leaves the context usable."""
    torch = pytest.importorskip("torch")
    ph, seq = list(cases())[0]
    p = M.Phantom.from_workload_phantom(ctx, ph)
    s = M.Sequence.from_workload_sequence(ctx, seq)
    out = torch.zeros(2 * s.n_adc, dtype=torch.float64, device="cuda")
    M.lib().mrsim_debug_fail_alloc(ctx.h, 0)  # the next device allocation: the maps
    with pytest.raises(M.MrsimError) as e:
        M.simulate(ctx, p, s, M.FP32, out=out)
    assert e.value.status == M.Status.ENOMEM
    M.lib().mrsim_debug_fail_alloc(ctx.h, -1)
    M.simulate(ctx, p, s, M.FP32, out=out)
    torch.cuda.synchronize()
    ctx.stream_status()
    assert rel_l2(out.cpu().numpy().view(np.complex128), oracle_mod.signal(ph, seq)) <= 2e-5


def test_train_maps_with_snapshots_and_resume(M, ctx, oracle_mod):
    """Snapshots inside and between the shaped pulses of a spin echo whose other pulses run as
    train maps, and a simulation resumed from a state in the middle of the sequence: every
    snapshot equals the oracle's state after that event, and the resumed signal the oracle's."""
    ph, seq = list(cases())[0]
    ev = seq.events
    per_tr = len(ev) // 16
    rf = np.flatnonzero(ev["rf_flip"] != 0)
    snaps = np.array(sorted({int(rf[5]), per_tr + 3, int(rf[len(rf) // 2]), 9 * per_tr - 1, len(ev) - 1}))
    p = M.Phantom.from_workload_phantom(ctx, ph)
    s = M.Sequence(ctx, ev, seq.gamma_hz_per_t, snapshots=snaps)
    out = np.zeros((len(snaps), ph.n, 3))
    for prec, tol in ((M.FP64, 1e-12), (M.FP32, 1e-4)):
        M.simulate(ctx, p, s, prec, snapshots=out)
        ctx.stream_status()
        for q, e in enumerate(snaps):
            _, st = oracle_mod.simulate(ph, ev[: e + 1], seq.gamma_hz_per_t, want_signal=False, want_state=True)
            assert np.max(np.abs(out[q] - st)) <= tol * max(1.0, np.abs(st).max()), (prec, q)
    # resume: the second half from the state after the first half
    half = 8 * per_tr
    _, mid = oracle_mod.simulate(ph, ev[:half], seq.gamma_hz_per_t, want_signal=False, want_state=True)
    ref2, _ = oracle_mod.simulate(ph, ev[half:], seq.gamma_hz_per_t, m_init=mid)
    s2 = M.Sequence(ctx, ev[half:], seq.gamma_hz_per_t)
    got2 = M.simulate(ctx, p, s2, M.FP64, state_in=mid.copy())
    assert rel_l2(got2, ref2) <= max(1e-12, phase_floor(ph, ev[half:], seq.gamma_hz_per_t))

