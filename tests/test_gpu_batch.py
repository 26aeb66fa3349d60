"""Batched simulation (many phantoms with their own sequences in one persistent launch, CUDA-graph
replay, autotuned launch shape) against the CPU oracle and against single-phantom launches."""
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


@pytest.fixture(scope="module")
def M(mrsim_lib):
    return mrsim_lib


@pytest.fixture(scope="module")
def ctx(M):
    c = M.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def torch():
    return pytest.importorskip("torch")


def small_batch(seed=0):
    """Uneven phantoms (0 .. 5000 spins) with their own sequences, including the paper's types."""
    rng = np.random.default_rng(seed)
    out = []
    sizes = [1, 37, 700, 2500, 5000, 0, 1200]
    for i, n in enumerate(sizes):
        ph = W.random_phantom(n, rng)
        ph.dw[:] = 2 * math.pi * rng.uniform(-50, 50, n)  # moderate phases: the 1e-12 float64 bar applies
        if i % 3 == 0:
            seq = W.flash(16, 16, 0.5, math.radians(rng.uniform(5, 90)), 6e-3, 3e-3, 10e-6)
        elif i % 3 == 1:
            seq = W.spin_echo(16, 8, 0.5, 12e-3, 30e-3, 10e-6, n_rf=24)
        else:
            seq = W.flash(16, 16, 0.5, 0.3, 5e-3, 2.5e-3, 10e-6, rf_spoil=True)
        out.append((ph, seq))
    return out


def make_batch(M, ctx, torch, pairs, prec):
    phs = [M.Phantom.from_workload_phantom(ctx, p) for p, _ in pairs]
    sqs = [M.Sequence.from_workload_sequence(ctx, s) for _, s in pairs]
    outs = [torch.zeros(max(2 * s.n_adc, 2), dtype=torch.float64, device="cuda") for s in sqs]
    b = M.Batch(ctx, phs, sqs, prec, outs)
    return b, phs, sqs, outs


def signals(outs, sqs):
    return [o.cpu().numpy()[: 2 * s.n_adc].view(np.complex128) for o, s in zip(outs, sqs)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_oracle(M, ctx, torch, oracle_mod, prec):
    pairs = small_batch()
    p = M.FP64 if prec == "fp64" else M.FP32
    tol = TOL64 if prec == "fp64" else TOL32
    refs = [oracle_mod.signal(ph, seq) for ph, seq in pairs]
    b, phs, sqs, outs = make_batch(M, ctx, torch, pairs, p)
    assert b.n_items > len(pairs) - 1
    for graph in (False, True, True):  # direct launch, graph capture, graph replay
        b.launch(graph=graph)
        torch.cuda.synchronize()
        ctx.stream_status()
        for got, ref in zip(signals(outs, sqs), refs):
            assert rel_l2(got, ref) <= tol


def test_batch_shapes_and_autotune(M, ctx, torch, oracle_mod):
    pairs = small_batch(seed=1)
    refs = [oracle_mod.signal(ph, seq) for ph, seq in pairs]
    b, phs, sqs, outs = make_batch(M, ctx, torch, pairs, M.FP32)
    for k, t in ((1, 32), (2, 96), (4, 128), (8, 64)):
        b.set_shape(k, t)
        b.launch(graph=True)
        torch.cuda.synchronize()
        for got, ref in zip(signals(outs, sqs), refs):
            assert rel_l2(got, ref) <= TOL32, (k, t)
    k, t = b.autotune()
    assert k in (1, 2, 4, 8) and 32 <= t <= 512
    b.launch()
    torch.cuda.synchronize()
    ctx.stream_status()
    for got, ref in zip(signals(outs, sqs), refs):
        assert rel_l2(got, ref) <= TOL32


def test_batch_rejects_host_output(M, ctx):
    ph = M.Phantom.from_workload_phantom(ctx, W.random_phantom(10, np.random.default_rng(2)))
    sq = M.Sequence.from_workload_sequence(ctx, W.flash(8, 8, 0.5, 0.3, 5e-3, 2.5e-3, 10e-6))
    host = np.zeros(2 * sq.n_adc)
    with pytest.raises(M.MrsimError) as e:
        M.Batch(ctx, [ph], [sq], M.FP32, [host])
    assert e.value.status == M.Status.EINVAL


def test_empty_batch(M, ctx):
    b = M.Batch(ctx, [], [], M.FP32, [])
    b.launch()
    b.launch(graph=True)
    ctx.stream_status()


@pytest.fixture(scope="module")
def c4():
    return W.config4()


def test_config4_batch_equals_single_launches(M, ctx, torch, oracle_mod, c4):
    """The 64-phantom batched workload (uneven 1e4..2e6 spins, FLASH/SE mix): one graph-replayed
    persistent launch equals 64 single-phantom launches, and the oracle on spin subsets."""
    ws = c4
    pairs = [(w.phantom, w.sequence) for w in ws]
    b, phs, sqs, outs = make_batch(M, ctx, torch, pairs, M.FP32)
    k, t = b.autotune()
    b.launch(graph=True)
    b.launch(graph=True)
    torch.cuda.synchronize()
    ctx.stream_status()
    got = signals(outs, sqs)
    for i in range(len(ws)):
        # same tiles as the batch: the same float32 arithmetic per spin; only the order in which
        # warps add into a block's window (float32 shared atomics) and blocks into the signal
        # (float64 atomics) differs, a few float32 roundings of the block sums
        single = M.simulate(ctx, phs[i], sqs[i], M.FP32, spins_per_thread=k, threads_per_block=t)
        assert rel_l2(got[i], single) <= 1e-6, i
    rng = np.random.default_rng(4)
    for i in (int(np.argmin([w.phantom.n for w in ws])), int(np.argmax([w.sequence.n_events for w in ws]))):
        w = ws[i]
        idx = np.sort(rng.choice(w.phantom.n, min(w.phantom.n, 300), replace=False))
        sub = w.phantom.subset(idx)
        ref = oracle_mod.signal(sub, w.sequence)
        ps = M.Phantom.from_workload_phantom(ctx, sub)
        assert rel_l2(M.simulate(ctx, ps, sqs[i], M.FP32), ref) <= TOL32


@pytest.fixture(scope="module")
def c4_samples(c4, oracle_mod):
    """The 4 smallest phantoms whole, every other phantom on a seeded 1 % sample of its tissue
    spins: (phantoms with M0 = 0 outside the samples, oracle signals of the samples)."""
    n = np.array([w.phantom.n for w in c4])
    whole = set(np.argsort(n)[:4].tolist())
    rng = np.random.default_rng(44)
    phs, refs = [], []
    for i, w in enumerate(c4):
        if i in whole:
            idx = np.arange(w.phantom.n)
        else:
            pool = np.nonzero(w.phantom.rho > 0)[0]
            idx = np.sort(rng.choice(pool, max(1, int(round(0.01 * w.phantom.n))), replace=False))
        ph = w.phantom
        rho = np.zeros_like(ph.rho)
        rho[idx] = ph.rho[idx]
        phs.append(W.Phantom(ph.x, ph.y, ph.z, rho, ph.t1, ph.t2, ph.dw))
        refs.append(oracle_mod.signal(ph.subset(idx), w.sequence))
    return phs, refs


# Bars on the C4 batch (FLASH phantoms, spin-echo phantoms): 2e-5 for float32 and the compensated
# precision, 1e-12 for float64.  The spin echoes keep transverse coherence over many TRs through
# 2 x 127 sub-pulse turns per TR; stepped sub-pulse by sub-pulse in float32 they drift up to 1.5e-4
# from float64, but their recurring shaped pulses run as train maps (one rounding of the composed
# map per pulse instead of one per sub-pulse), which brings every C4 phantom within 5e-6 of
# float64 on the full phantom.
C4_TOL = {"fp64": (1e-12, 1e-12), "fp32": (2e-5, 2e-5), "fp32_kahan": (2e-5, 2e-5)}


@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp32_kahan"])
def test_config4_batch_graph_against_oracle(M, ctx, torch, c4, c4_samples, prec):
    """The 64-phantom batch through the graph-replayed persistent launch itself, against the
    oracle: the 4 smallest phantoms whole, every other phantom on a seeded 1 % sample of its
    tissue spins.  The batch holds all 64 phantoms at full size, with M0 = 0 outside each sample
    (such spins stay at (0, 0, 0) and add exact zeros), so the samples run in the batch's own work
    items and launch shape."""
    phs_m, refs = c4_samples
    p = {"fp64": M.FP64, "fp32": M.FP32, "fp32_kahan": M.FP32_KAHAN}[prec]
    tol_flash, tol_se = C4_TOL[prec]
    b, phs, sqs, outs = make_batch(M, ctx, torch, list(zip(phs_m, [w.sequence for w in c4])), p)
    if p != M.FP64:
        b.autotune()  # the benchmark's batch tuning
    b.launch(graph=True)  # capture
    b.launch(graph=True)  # replay
    torch.cuda.synchronize()
    ctx.stream_status()
    worst = 0.0
    for i, (g, r) in enumerate(zip(signals(outs, sqs), refs)):
        assert np.linalg.norm(r) > 0, i
        tol = tol_se if c4[i].sequence.name.startswith("se") else tol_flash
        e = rel_l2(g, r)
        worst = max(worst, e)
        assert e <= tol, (i, c4[i].name, e)
    if p == M.FP32_KAHAN:
        assert worst <= 1e-10
