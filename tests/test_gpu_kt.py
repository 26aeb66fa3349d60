"""K-t formalism on the GPU (mrsim_kt_simulate) against the oracle (oracle/kt.py, §4.2).

Inputs are seeded (workloads.kt_dictionary / kt_fingerprint_sequence / kt_random_sequence):
dictionaries over T1, T2, B1 and off-resonance, a fingerprinting-style train and random step
lists with order shifts of -2..2.  Tolerances: float64 1e-12, float32 2e-5 (relative L2).
"""
import math

import numpy as np
import pytest

from oracle import kt as ORK
from paper_1305_6861_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="module")
def M(mrsim_lib):
    return mrsim_lib


@pytest.fixture(scope="module")
def ctx(M):
    c = M.Context(0)
    yield c
    c.close()


def both(M, ctx, d, steps, K):
    ref = ORK.simulate(d.t1, d.t2, d.b1, d.df, steps, K)
    g64 = M.kt_simulate(ctx, d.t1, d.t2, steps, K, b1=d.b1, df=d.df, precision=M.FP64)
    g32 = M.kt_simulate(ctx, d.t1, d.t2, steps, K, b1=d.b1, df=d.df, precision=M.FP32)
    return ref, g64, g32


@pytest.mark.parametrize("K", [100, 127])  # 127 fills 4 slots per lane: the kernel's fast step
def test_fingerprint_dictionary(M, ctx, K):
    rng = np.random.default_rng(1300)
    d = W.kt_dictionary(67, rng)  # 17 blocks of 4 ensembles, ragged
    steps = W.kt_fingerprint_sequence(300, rng)
    ref, g64, g32 = both(M, ctx, d, steps, K)
    assert rel_l2(g64, ref) <= TOL64
    assert rel_l2(g32, ref) <= TOL32


@pytest.mark.parametrize("K", [0, 5, 31, 32, 33, 64, 130, 255])
def test_random_steps_and_truncation(M, ctx, K):
    rng = np.random.default_rng(1400 + K)
    d = W.kt_dictionary(9, rng)
    steps = W.kt_random_sequence(120, rng, max_shift=2)
    ref, g64, g32 = both(M, ctx, d, steps, K)
    assert rel_l2(g64, ref) <= TOL64, K
    assert rel_l2(g32, ref) <= TOL32, K


def test_kt_matches_isochromat_path(M, ctx):
    """N isochromats over one gradient cycle through the spin-based kernel equal the K-t a_0 (§4.2,
    discrete orthogonality): the library's two methods agree with each other."""
    rng = np.random.default_rng(1500)
    n_iso, dk = 64, 5.0
    t1, t2, b1, df = 0.9, 0.11, 1.1, 12.0
    x = np.arange(n_iso) / (n_iso * dk)
    ph = W.Phantom(x, np.zeros(n_iso), np.zeros(n_iso), np.full(n_iso, 1.0 / n_iso), np.full(n_iso, t1),
                   np.full(n_iso, t2), np.full(n_iso, 2 * math.pi * df))
    steps = W.kt_random_sequence(14, rng, max_shift=2)
    steps["sample"][-1] = 1
    ev = W.make_events([(s["tau"], s["shift"] * dk / (W.GAMMA_BAR * s["tau"]) if s["tau"] > 0 else 0.0, 0.0, 0.0,
                         b1 * s["alpha"], s["phi"], int(s["sample"]), s["adc_phase"]) for s in steps])
    keep = ~((steps["tau"] == 0) & (steps["shift"] != 0))  # a moment needs an interval
    steps, ev = steps[keep], ev[keep]
    spins = M.simulate(ctx, M.Phantom.from_workload_phantom(ctx, ph), M.Sequence(ctx, ev, W.GAMMA_BAR), M.FP64)
    kt = M.kt_simulate(ctx, [t1], [t2], steps, 40, b1=[b1], df=[df], precision=M.FP64)[0]
    assert rel_l2(kt, spins) <= 1e-12


def test_device_buffers(M, ctx):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1600)
    d = W.kt_dictionary(40, rng)
    steps = W.kt_fingerprint_sequence(50, rng)
    ref = ORK.simulate(d.t1, d.t2, d.b1, d.df, steps, 60)
    dev = [torch.from_numpy(a.copy()).cuda() for a in (d.t1, d.t2, d.b1, d.df)]
    out = torch.zeros(d.n * 2 * 50, dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        M.kt_simulate(ctx, dev[0], dev[1], steps, 60, b1=dev[2], df=dev[3], precision=M.FP32, stream=st, out=out)
    st.synchronize()
    got = out.cpu().numpy().view(np.complex128).reshape(d.n, 50)
    assert rel_l2(got, ref) <= TOL32


def test_invalid_kt_inputs(M, ctx):
    d = W.kt_dictionary(4, np.random.default_rng(1))
    steps = W.kt_fingerprint_sequence(10, np.random.default_rng(2))
    bad = steps.copy()
    bad["tau"][3] = np.nan
    for st, K in ((bad, 10), (steps, M.KT_MAX_ORDER + 1), (steps, -1)):
        with pytest.raises(M.MrsimError) as e:
            M.kt_simulate(ctx, d.t1, d.t2, st, K)
        assert e.value.status == M.Status.EINVAL
    big = steps.copy()
    big["shift"][2] = 65
    with pytest.raises(M.MrsimError):
        M.kt_simulate(ctx, d.t1, d.t2, big, 10)
    t1 = d.t1.copy()
    t1[2] = 0.0
    with pytest.raises(M.MrsimError) as e:
        M.kt_simulate(ctx, t1, d.t2, steps, 10)
    assert "ensemble 2" in str(e.value)
    rc = M.lib().mrsim_kt_simulate(ctx.h, d.n, M._ptr(d.t1), M._ptr(d.t2), None, None, steps.shape[0], M._ptr(steps),
                                   10, M.FP32, None, M._ptr(np.zeros(2 * d.n * 20)), 11)
    assert rc == M.Status.EINVAL


def test_full_size_fingerprint_dictionary_sampled(M, ctx):
    """The benchmark's workload at full size, in its launch configuration (65 536 ensembles ×
    1001 steps, K = 127, the seeded dictionary of the benchmark): both precisions on the GPU,
    sampled ensembles against the oracle one by one (every ensemble is independent)."""
    rng = np.random.default_rng(W.SEED_BASE + 6)
    d = W.kt_dictionary(65536, rng)
    steps = W.kt_fingerprint_sequence(1000, rng)
    K = 127
    g64 = M.kt_simulate(ctx, d.t1, d.t2, steps, K, b1=d.b1, df=d.df, precision=M.FP64)
    g32 = M.kt_simulate(ctx, d.t1, d.t2, steps, K, b1=d.b1, df=d.df, precision=M.FP32)
    pick = np.sort(np.random.default_rng(7).choice(d.n, 12, replace=False))
    pick = np.concatenate([[0], pick, [d.n - 1]])
    for i in pick:
        ref = ORK.simulate_one(d.t1[i], d.t2[i], d.b1[i], d.df[i], steps, K)
        assert rel_l2(g64[i], ref) <= TOL64, i
        assert rel_l2(g32[i], ref) <= TOL32, i
