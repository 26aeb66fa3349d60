"""Adjoint (backward-in-time) gradients on the GPU against the oracle's forward-mode gradient and
central finite differences (h = 1e-4 relative, float64), and the autograd.Function."""
import math

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="module")
def torch():
    return pytest.importorskip("torch")


@pytest.fixture(scope="module")
def M(mrsim_lib):
    return mrsim_lib


@pytest.fixture(scope="module")
def ctx(M):
    c = M.Context(0)
    yield c
    c.close()


def shaped_case(seed, n_sp, n_rf=16, n_tr=3, n_read=8):
    rng = np.random.default_rng(seed)
    ph = W.random_phantom(n_sp, rng, inf_frac=0.1)
    ph.dw[:] = 2 * math.pi * rng.uniform(-50, 50, n_sp)
    base = W.sinc_pulse(0.6, n_rf, 4.0)
    rows, params = [], []
    for tr in range(n_tr):
        for i, a in enumerate(base):
            rows.append((20e-6, 0, 0, 2e-3, float(a), 0.3 * tr, 0, 0.0))
            params.append(i)
        rows.append((1e-3, -1e-3, 2e-3 * (tr - 1), 0, 0, 0, 0, 0.0))
        rows += [(20e-6, 2e-3, 0, 0, 0, 0, 1, 0.3 * tr)] * n_read
        params += [-1] * (1 + n_read)
        rows.append((4e-3, 0, 0, 0, 0, 0, 0, 0.0))
        params.append(-1)
    ev = W.make_events(rows)
    rf = np.array(base) * rng.uniform(0.8, 1.2, n_rf)
    return ph, ev, np.array(params, dtype=np.int32), rf, rng


def gpu_grads(M, ctx, torch, ph, ev, params, rf, h, ckpt=64, precision=None):
    adj = M.Adjoint(ctx, ev, W.GAMMA_BAR, params, len(rf), ckpt_every=ckpt)
    if precision is not None:
        adj.set_precision(precision)
    P = M.Phantom.from_workload_phantom(ctx, ph)
    dev = torch.device("cuda:0")
    rfd = torch.from_numpy(np.asarray(rf, dtype=np.float64)).to(dev)
    sig = torch.zeros(2 * adj.n_adc, dtype=torch.float64, device=dev)
    adj.forward(P, rfd, sig)
    hd = torch.from_numpy(np.ascontiguousarray(np.asarray(h, dtype=np.complex128)).view(np.float64)).to(dev)
    out = [torch.zeros(ph.n, dtype=torch.float64, device=dev) for _ in range(3)]
    drf = torch.zeros(len(rf), dtype=torch.float64, device=dev)
    adj.backward(P, hd, rfd, *out, drf)
    torch.cuda.synchronize()
    ctx.stream_status()
    return sig.cpu().numpy().view(np.complex128), [o.cpu().numpy() for o in out], drf.cpu().numpy()


# up to 256 RF parameters each thread sums its RF gradients in local memory, beyond that every
# pulse reduces over the warp; up to 1024 the forward pass is the library's forward kernel on a
# parametric program, beyond that the adjoint's own forward kernel.  `n_par` declares that many
# learnable flips (the pulse uses the first n_rf; the others get zero gradient), so every path
# runs on the same well-conditioned sequences.
@pytest.mark.parametrize("seed,n_sp,ckpt,n_rf,n_par", [(0, 40, 64, 16, 16), (1, 300, 7, 16, 16), (2, 1, 1, 16, 16),
                                                      (3, 129, 128, 16, 16), (4, 70, 64, 300, 300),
                                                      (5, 33, 32, 16, 256), (6, 20, 64, 16, 1100)])
def test_adjoint_matches_oracle_gradient(M, ctx, torch, oracle_mod, seed, n_sp, ckpt, n_rf, n_par):
    ph, ev, params, rf, rng = shaped_case(seed, n_sp, n_rf=n_rf, n_tr=3 if n_rf <= 16 else 2)
    rf = np.concatenate([rf, rng.uniform(-1.0, 1.0, n_par - n_rf)])
    sig_ref = oracle_mod.simulate_rf(ph, ev, W.GAMMA_BAR, params, rf)
    target = oracle_mod.simulate_rf(ph, ev, W.GAMMA_BAR, params, rf * 1.1) * 0.9
    h = 2 * (sig_ref - target)
    g_rho, g_t1, g_t2, g_rf = oracle_mod.gradient(ph, ev, W.GAMMA_BAR, h, params, rf, list(range(len(rf))))
    sig, (a_rho, a_t1, a_t2), a_rf = gpu_grads(M, ctx, torch, ph, ev, params, rf, h, ckpt)
    assert rel(sig, sig_ref) <= 1e-12
    assert rel(a_rho, g_rho) <= 1e-10
    assert rel(a_t1, g_t1) <= 1e-10
    assert rel(a_t2, g_t2) <= 1e-10
    assert rel(a_rf, g_rf) <= 1e-10


def test_adjoint_config5_full_size(M, ctx, torch, oracle_mod):
    """C5 (128² spins, 256 learnable sub-pulses, 49 408 events): the adjoint against the oracle's
    gradient on sampled spins (per-spin gradients depend only on h and the spin) and against
    central differences of the GPU float64 forward for sampled RF coordinates."""
    w, tgt, rf0 = W.config5()
    ev = w.sequence.events
    params = np.full(len(ev), -1, dtype=np.int32)
    idx = W.rf_event_index(w.sequence)
    params[idx] = np.tile(np.arange(len(rf0), dtype=np.int32), idx.size // len(rf0))
    dev = torch.device("cuda:0")
    adj = M.Adjoint(ctx, ev, W.GAMMA_BAR, params, len(rf0), ckpt_every=64)
    P = M.Phantom.from_workload_phantom(ctx, w.phantom)
    PT = M.Phantom.from_workload_phantom(ctx, tgt)
    rfd = torch.from_numpy(rf0.copy()).to(dev)
    sig = torch.zeros(2 * adj.n_adc, dtype=torch.float64, device=dev)
    tsig = torch.zeros_like(sig)
    adj.forward(PT, rfd, tsig)
    adj.forward(P, rfd, sig)
    torch.cuda.synchronize()
    # the adjoint's forward equals the optimised forward path on the same sequence
    seq = M.Sequence.from_workload_sequence(ctx, w.sequence)
    s_fast = M.simulate(ctx, P, seq, M.FP64)
    s = sig.cpu().numpy().view(np.complex128)
    assert rel(s, s_fast) <= 1e-12
    t = tsig.cpu().numpy().view(np.complex128)
    h = 2 * (s - t)
    hd = torch.from_numpy(np.ascontiguousarray(h).view(np.float64)).to(dev)
    out = [torch.zeros(w.phantom.n, dtype=torch.float64, device=dev) for _ in range(3)]
    drf = torch.zeros(len(rf0), dtype=torch.float64, device=dev)
    adj.backward(P, hd, rfd, *out, drf)
    torch.cuda.synchronize()
    ctx.stream_status()
    a_rho, a_t1, a_t2 = [o.cpu().numpy() for o in out]
    a_rf = drf.cpu().numpy()
    sel = np.sort(np.random.default_rng(5).choice(w.phantom.n, 256, replace=False))
    sub = w.phantom.subset(sel)
    g_rho, g_t1, g_t2, _ = oracle_mod.gradient(sub, ev, W.GAMMA_BAR, h, params, rf0)
    assert rel(a_rho[sel], g_rho) <= 1e-9
    assert rel(a_t1[sel], g_t1) <= 1e-9
    assert rel(a_t2[sel], g_t2) <= 1e-9
    # central differences of L = |s - t|² in the RF coordinates, GPU float64 forward
    def loss(rfv):
        adj.forward(P, torch.from_numpy(rfv).to(dev), sig)
        torch.cuda.synchronize()
        return float(np.sum(np.abs(sig.cpu().numpy().view(np.complex128) - t) ** 2))
    for p in (0, 100, 128, 200):
        step = 1e-4 * max(abs(rf0[p]), 1e-3)
        rp, rm = rf0.copy(), rf0.copy()
        rp[p] += step
        rm[p] -= step
        fd = (loss(rp) - loss(rm)) / (2 * step)
        assert abs(fd - a_rf[p]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(a_rf).max()), (p, fd, a_rf[p])


def test_autograd_function(M, ctx, torch, oracle_mod):
    from paper_1305_6861_gb300 import autograd as AG

    ph, ev, params, rf, rng = shaped_case(9, 24)
    dev = torch.device("cuda:0")
    adj = M.Adjoint(ctx, ev, W.GAMMA_BAR, params, len(rf))
    geom = [torch.from_numpy(a).to(dev) for a in (ph.x, ph.y, ph.z, ph.dw)]
    ph.t1[:] = np.minimum(ph.t1, 3.0)
    ph.t2[:] = np.minimum(ph.t2, 0.5)
    leaf = [torch.from_numpy(a.copy()).to(dev).requires_grad_(True) for a in (ph.rho, ph.t1, ph.t2, rf)]
    target = torch.from_numpy(np.ascontiguousarray(oracle_mod.simulate_rf(ph, ev, W.GAMMA_BAR, params, rf * 1.05))
                              .view(np.float64).reshape(-1, 2)).to(dev)
    s = AG.signal(adj, *geom, *leaf)
    loss = ((s - target) ** 2).sum()
    loss.backward()
    h = 2 * (s.detach().cpu().numpy().view(np.complex128).ravel() - target.cpu().numpy().view(np.complex128).ravel())
    g = oracle_mod.gradient(ph, ev, W.GAMMA_BAR, h, params, rf, list(range(len(rf))))
    for got, want in zip([t.grad.cpu().numpy() for t in leaf], g):
        assert rel(got, want) <= 1e-10
    # torch's own numerical check on a few coordinates
    small = [t.detach()[:3].clone().requires_grad_(True) for t in leaf[:3]] + [leaf[3].detach().clone().requires_grad_(True)]
    geom3 = [g_[:3].contiguous() for g_ in geom]
    f = lambda a, b, c, d: AG.signal(adj, *geom3, a, b, c, d)
    assert torch.autograd.gradcheck(f, tuple(small), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_allocation_failures_in_adjoint(M, torch, oracle_mod):
    """Each device allocation of adjoint creation and of the first forward pass (the checkpoint
    store) fails in turn through the allocation-failure hook: the call returns MRSIM_ENOMEM and
    the context stays usable; once the hook stops firing, the same calls give the oracle's
    signal."""
    ph, ev, params, rf, _ = shaped_case(31, 300)
    L = M.lib()
    c = M.Context(0)
    try:
        P = M.Phantom.from_workload_phantom(c, ph)
        dev = torch.device("cuda:0")
        rfd = torch.from_numpy(np.asarray(rf, dtype=np.float64)).to(dev)
        failed = 0
        for after in range(16):
            assert L.mrsim_debug_fail_alloc(c.h, after) == 0
            adj = None
            try:
                adj = M.Adjoint(c, ev, W.GAMMA_BAR, params, len(rf), ckpt_every=16)
                sig = torch.zeros(2 * adj.n_adc, dtype=torch.float64, device=dev)
                adj.forward(P, rfd, sig)
                torch.cuda.synchronize()
                c.stream_status()
            except M.MrsimError as e:
                assert e.status == M.Status.ENOMEM, e
                failed += 1
                continue
            finally:
                if adj is not None:
                    adj.close()
            break
        else:
            pytest.fail("the hook never stopped firing")
        L.mrsim_debug_fail_alloc(c.h, -1)
        # events, pulse specs, rotation tables, classes, demodulation, the forward program, checkpoints
        assert failed >= 6
        assert rel(sig.cpu().numpy().view(np.complex128), oracle_mod.simulate_rf(ph, ev, W.GAMMA_BAR, params, rf)) <= 1e-12
        P.close()
    finally:
        c.close()


@pytest.mark.parametrize("seed,n_sp,ckpt,host", [(10, 150, 64, True), (11, 37, 5, False), (12, 1, 0, True)])
def test_simulate_adjoint_one_shot(M, ctx, torch, oracle_mod, seed, n_sp, ckpt, host):
    """mrsim_simulate_adjoint on a loaded sequence: every pulse's flip is a learnable parameter (in
    event order); host or device buffers; against the oracle's forward-mode gradient at the
    adjoint's bar; a float32 precision is refused (the gradients are float64)."""
    ph, ev, _, _, rng = shaped_case(seed, n_sp)
    flips = ev["rf_flip"]
    params = np.full(len(ev), -1, dtype=np.int32)
    pulses = np.nonzero(flips != 0)[0]
    params[pulses] = np.arange(pulses.size, dtype=np.int32)
    rf = flips[pulses].copy()
    sig = oracle_mod.simulate_rf(ph, ev, W.GAMMA_BAR, params, rf)
    h = 2 * (sig - 0.8 * sig[::-1])
    g = oracle_mod.gradient(ph, ev, W.GAMMA_BAR, h, params, rf, list(range(rf.size)))
    P = M.Phantom.from_workload_phantom(ctx, ph)
    seq = M.Sequence(ctx, ev, W.GAMMA_BAR)
    assert M.lib().mrsim_sequence_num_pulses(seq.h) == pulses.size
    if host:
        got = M.simulate_adjoint(ctx, P, seq, h, ckpt_every=ckpt)
    else:
        dev = torch.device("cuda:0")
        hd = torch.from_numpy(np.ascontiguousarray(h).view(np.float64).copy()).to(dev)
        outs = [torch.zeros(ph.n, dtype=torch.float64, device=dev) for _ in range(3)]
        outs.append(torch.zeros(pulses.size, dtype=torch.float64, device=dev))
        M.simulate_adjoint(ctx, P, seq, hd, ckpt_every=ckpt, outs=outs)
        got = [o.cpu().numpy() for o in outs]
    for a, b in zip(got, g):
        assert rel(a, b) <= 1e-10
    # without RF gradients, only the spin parameters
    d_rho, d_t1, d_t2, d_rf = M.simulate_adjoint(ctx, P, seq, h, rf=False)
    assert d_rf is None and rel(d_rho, g[0]) <= 1e-10 and rel(d_t2, g[2]) <= 1e-10
    with pytest.raises(M.MrsimError) as e:
        M.simulate_adjoint(ctx, P, seq, h, precision=M.FP32)
    assert e.value.status == M.Status.EUNSUPPORTED
    # the compensated precision of the same call
    gk = M.simulate_adjoint(ctx, P, seq, h, precision=M.FP32_KAHAN, ckpt_every=ckpt)
    for a, b in zip(gk, g):
        assert rel(a, b) <= 1e-10



@pytest.mark.parametrize("seed,n_sp,ckpt,n_rf,n_par", [(20, 300, 64, 16, 16), (21, 129, 7, 16, 256),
                                                      (22, 40, 64, 16, 1100)])
def test_compensated_adjoint_matches_oracle_gradient(M, ctx, torch, oracle_mod, seed, n_sp, ckpt, n_rf, n_par):
    """The adjoint recursion in the compensated precision (double-float pairs on the FP32 pipe):
    forward signal and gradients in M0, T1, T2 and the learnable flips against the oracle at the
    float64 adjoint's bars, on every path (local / warp-reduced RF gradients, library forward /
    the adjoint's own forward)."""
    ph, ev, params, rf, rng = shaped_case(seed, n_sp, n_rf=n_rf)
    rf = np.concatenate([rf, rng.uniform(-1.0, 1.0, n_par - n_rf)])
    sig_ref = oracle_mod.simulate_rf(ph, ev, W.GAMMA_BAR, params, rf)
    h = 2 * (sig_ref - 0.9 * oracle_mod.simulate_rf(ph, ev, W.GAMMA_BAR, params, rf * 1.1))
    g = oracle_mod.gradient(ph, ev, W.GAMMA_BAR, h, params, rf, list(range(len(rf))))
    sig, (a_rho, a_t1, a_t2), a_rf = gpu_grads(M, ctx, torch, ph, ev, params, rf, h, ckpt, M.FP32_KAHAN)
    assert rel(sig, sig_ref) <= 1e-11
    for a, b in zip((a_rho, a_t1, a_t2, a_rf), g):
        assert rel(a, b) <= 1e-10


def test_compensated_adjoint_config5(M, ctx, torch, oracle_mod):
    """C5 in the compensated precision: signal and spin gradients against the float64 adjoint on
    the full phantom, and a sampled spin set against the oracle's gradient."""
    w, tgt, rf0 = W.config5()
    ev = w.sequence.events
    params = np.full(len(ev), -1, dtype=np.int32)
    idx = W.rf_event_index(w.sequence)
    params[idx] = np.tile(np.arange(len(rf0), dtype=np.int32), idx.size // len(rf0))
    h = np.random.default_rng(5).normal(size=w.sequence.n_adc) * (1 + 1j)
    res = {}
    for prec in (M.FP64, M.FP32_KAHAN):
        res[prec] = gpu_grads(M, ctx, torch, w.phantom, ev, params, rf0, h, 64, prec)
    s64, g64, r64 = res[M.FP64]
    sk, gk, rk = res[M.FP32_KAHAN]
    assert rel(sk, s64) <= 1e-11
    for a, b in zip(gk, g64):
        assert rel(a, b) <= 1e-10
    assert rel(rk, r64) <= 1e-10
    sel = np.sort(np.random.default_rng(6).choice(w.phantom.n, 300, replace=False))
    go = oracle_mod.gradient(w.phantom.subset(sel), ev, W.GAMMA_BAR, h, params, rf0, [])
    for a, b in zip(gk, go[:3]):
        assert rel(a[sel], b) <= 1e-10
