"""Receive coils (mrsim_simulate_coils) against the oracle's coil weighting (Eq. 3.25).

Sensitivities are synthetic: n coils on a ring around the object, each a Gaussian magnitude
profile of the distance to the coil with a phase that grows along the ring (the usual shape of
array-coil maps), plus random complex weights for the stress sequences.  Tolerances as for the
single-coil path: relative L2 over all coils, float32 ≤ 2e-5, float64 ≤ 1e-12 (or the phase
floor of the stress sequences).
"""
import math

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def ring_coils(ph, n_coils, radius=0.3, width=0.25):
    ang = 2 * math.pi * np.arange(n_coils) / n_coils
    cx, cy = radius * np.cos(ang), radius * np.sin(ang)
    d2 = (ph.x[None, :] - cx[:, None]) ** 2 + (ph.y[None, :] - cy[:, None]) ** 2
    return np.exp(-d2 / width**2) * np.exp(1j * (ang[:, None] + 4.0 * (ph.x[None, :] * np.cos(ang)[:, None])))


def phase_floor(ph, seq):
    ev = seq.events
    g = 2 * math.pi * seq.gamma_hz_per_t
    th = (g * (np.abs(ev["gx"]) * np.abs(ph.x).max() + np.abs(ev["gy"]) * np.abs(ph.y).max()
               + np.abs(ev["gz"]) * np.abs(ph.z).max()) + np.abs(ph.dw).max()) * ev["dt"]
    return max(TOL64, 4 * 2.0**-53 * float(np.sqrt(np.sum(th**2))))


@pytest.fixture(scope="module")
def M(mrsim_lib):
    return mrsim_lib


@pytest.fixture(scope="module")
def ctx(M):
    c = M.Context(0)
    yield c
    c.close()


def run(M, ctx, ph, seq, sens, prec):
    p = M.Phantom.from_workload_phantom(ctx, ph)
    s = M.Sequence.from_workload_sequence(ctx, seq)
    out = M.simulate_coils(ctx, p, s, sens, prec)
    ctx.stream_status()
    return out


@pytest.mark.parametrize("n_coils", [1, 3, 4, 8])
def test_config1_coils_parity(M, ctx, oracle_mod, n_coils):
    w = W.config1()
    sens = ring_coils(w.phantom, n_coils)
    ref = oracle_mod.simulate_coils(w.phantom, w.sequence.events, w.sequence.gamma_hz_per_t, sens)
    assert rel_l2(run(M, ctx, w.phantom, w.sequence, sens, M.FP64), ref) <= TOL64
    assert rel_l2(run(M, ctx, w.phantom, w.sequence, sens, M.FP32), ref) <= TOL32


@pytest.mark.parametrize("seed,n_coils", [(0, 2), (1, 5), (2, 8)])
def test_random_sequences_coils_parity(M, ctx, oracle_mod, seed, n_coils):
    rng = np.random.default_rng(800 + seed)
    ph = W.random_phantom(1500 + 333 * seed, rng)  # several blocks, ragged tail
    seq = W.random_sequence(1200, rng, runs=True)
    sens = rng.normal(size=(n_coils, ph.n)) + 1j * rng.normal(size=(n_coils, ph.n))
    ref = oracle_mod.simulate_coils(ph, seq.events, seq.gamma_hz_per_t, sens)
    assert rel_l2(run(M, ctx, ph, seq, sens, M.FP64), ref) <= phase_floor(ph, seq)
    assert rel_l2(run(M, ctx, ph, seq, sens, M.FP32), ref) <= TOL32


def test_long_runs_cross_the_sample_window(M, ctx, oracle_mod):
    """256-sample readouts with 8 coils exceed one window (128 samples in float32, 32 in float64)."""
    w = W.config2(n=16, iso=2)
    rng = np.random.default_rng(5)
    ph = w.phantom.subset(np.sort(rng.choice(w.phantom.n, size=min(w.phantom.n, 200), replace=False)))
    ev = w.sequence.events
    seq = W.Sequence(ev, w.sequence.gamma_hz_per_t)
    long_seq = W.spin_echo(256, 4, 0.5, 50e-3, 80e-3, 10e-6)
    sens = ring_coils(ph, 8)
    for sq in (seq, long_seq):
        ref = oracle_mod.simulate_coils(ph, sq.events, sq.gamma_hz_per_t, sens)
        assert rel_l2(run(M, ctx, ph, sq, sens, M.FP64), ref) <= TOL64
        assert rel_l2(run(M, ctx, ph, sq, sens, M.FP32), ref) <= TOL32


def test_homogeneous_coil_is_the_plain_signal(M, ctx):
    w = W.config1()
    p = M.Phantom.from_workload_phantom(ctx, w.phantom)
    s = M.Sequence.from_workload_sequence(ctx, w.sequence)
    ones = np.ones((1, w.phantom.n), dtype=np.complex128)
    # float32: the two paths sum in different orders and launch shapes; each is within TOL32 of
    # the exact signal, so they agree to TOL32
    for prec, tol in ((M.FP64, 1e-13), (M.FP32, TOL32)):
        plain = M.simulate(ctx, p, s, prec)
        coil = M.simulate_coils(ctx, p, s, ones, prec)[0]
        assert rel_l2(coil, plain) <= tol


def test_device_buffers(M, ctx, oracle_mod):
    torch = pytest.importorskip("torch")
    w = W.config1()
    sens = ring_coils(w.phantom, 4)
    ref = oracle_mod.simulate_coils(w.phantom, w.sequence.events, w.sequence.gamma_hz_per_t, sens)
    p = M.Phantom.from_workload_phantom(ctx, w.phantom)
    s = M.Sequence.from_workload_sequence(ctx, w.sequence)
    ds = torch.from_numpy(sens.view(np.float64).reshape(-1).copy()).cuda()
    out = torch.zeros(4 * 2 * s.n_adc, dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        M.simulate_coils(ctx, p, s, ds, M.FP32, stream=st, out=out)
    st.synchronize()
    got = out.cpu().numpy().view(np.complex128).reshape(4, -1)
    assert rel_l2(got, ref) <= TOL32


def test_invalid_coil_inputs(M, ctx):
    w = W.config1()
    p = M.Phantom.from_workload_phantom(ctx, w.phantom)
    s = M.Sequence.from_workload_sequence(ctx, w.sequence)
    for n_coils in (0, M.MAX_COILS + 1):
        sens = np.ones((max(n_coils, 1), w.phantom.n), dtype=np.complex128)
        rc = M.lib().mrsim_simulate_coils(ctx.h, p.h, s.h, M.FP32, None, n_coils, M._ptr(sens),
                                          M._ptr(np.zeros(2 * s.n_adc * max(n_coils, 1))), s.n_adc)
        assert rc == M.Status.EINVAL
    bad = np.ones((2, w.phantom.n), dtype=np.complex128)
    bad[1, 17] = np.nan
    with pytest.raises(M.MrsimError) as e:
        M.simulate_coils(ctx, p, s, bad, M.FP32)
    assert e.value.status == M.Status.EINVAL
    rc = M.lib().mrsim_simulate_coils(ctx.h, p.h, s.h, M.FP32, None, 1, M._ptr(bad[:1].copy()),
                                      M._ptr(np.zeros(2 * s.n_adc)), s.n_adc + 1)
    assert rc == M.Status.EINVAL
