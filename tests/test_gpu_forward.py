"""Forward-simulation parity of the CUDA library (through the C-ABI) against the CPU oracle.

Tolerances (relative L2 error of the complex signal): 1e-12 for the float64 path, 2e-5 for
the float32 path.  Sizes span several thread blocks with a ragged tail; the full-size
workloads are checked on spin subsets (the signal is additive over spins, §5.3.2) in the
launch shape the benchmark uses, plus properties that hold at any size.
"""
import math
import os

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def fp64_phase_tolerance(ph, seq):
    """float64 floor for sequences with very large per-event phases (stress sequences).

    An event turns a spin by θ = (γ G·x + Δω)·Δt; each implementation (oracle included)
    represents θ with a relative rounding of ε = 2^-53, i.e. an absolute phase error of
    about ε·|θ| per event, independently per event.  The signal error relative to the
    signal is then of order ε·sqrt(Σ_e θ_e²) over the largest phases; 4x covers both
    sides and the sin/cos evaluation.  For the paper's workloads this is below 1e-12.
    """
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


def run(M, ctx, ph, seq, prec, **kw):
    p = M.Phantom.from_workload_phantom(ctx, ph)
    s = M.Sequence.from_workload_sequence(ctx, seq)
    out = M.simulate(ctx, p, s, prec, **kw)
    ctx.stream_status()
    return out


def test_config1_parity(M, ctx, oracle_mod):
    w = W.config1()
    ref = oracle_mod.signal(w)
    assert rel_l2(run(M, ctx, w.phantom, w.sequence, M.FP64), ref) <= TOL64
    assert rel_l2(run(M, ctx, w.phantom, w.sequence, M.FP32), ref) <= TOL32


@pytest.mark.parametrize("seed", range(4))
def test_random_sequences_parity(M, ctx, oracle_mod, seed):
    rng = np.random.default_rng(500 + seed)
    ph = W.random_phantom(1000 + 777 * seed, rng)  # several blocks, ragged tail
    seq = W.random_sequence(1500, rng, runs=True)
    ref, ref_state = oracle_mod.simulate(ph, seq.events, seq.gamma_hz_per_t, want_state=True)
    st64 = np.zeros((ph.n, 3))
    s64 = run(M, ctx, ph, seq, M.FP64, state_out=st64)
    tol = fp64_phase_tolerance(ph, seq)
    assert rel_l2(s64, ref) <= tol
    assert np.max(np.abs(st64 - ref_state)) <= tol * max(1.0, np.abs(ref_state).max())
    st32 = np.zeros((ph.n, 3))
    s32 = run(M, ctx, ph, seq, M.FP32, state_out=st32)
    assert rel_l2(s32, ref) <= TOL32
    assert np.max(np.abs(st32 - ref_state)) <= 1e-4


def _inline_phase_sequence(rng, cycles, n_rep=40):
    """Unique free-precession intervals (so they compile to inline precessions) whose largest
    k·x term is about `cycles` cycles at the edge of a 0.5 m field of view, each followed by one
    sample, with a hard pulse every 8 intervals."""
    rows = [(0.0, 0.0, 0.0, 0.0, math.pi / 2, 0.3, 0, 0.0)]
    kmax = cycles / 0.25  # cycles/m
    for i in range(n_rep):
        dt = rng.uniform(1e-4, 2e-3)
        g = rng.uniform(-1, 1, 3) * kmax / (W.GAMMA_BAR * dt)
        rows.append((dt, *g, 0.0, 0.0, 0, 0.0))
        rows.append((1e-5, 0.0, 0.0, 0.0, 0.0, 0.0, 1, rng.uniform(0, 2 * math.pi)))
        if i % 8 == 7:
            rows.append((0.0, 0.0, 0.0, 0.0, rng.uniform(0.2, 1.0), rng.uniform(0, 2 * math.pi), 0, 0.0))
    return W.Sequence(W.make_events(rows), W.GAMMA_BAR)


@pytest.mark.parametrize("cycles", [300.0, 5.0e6])
@pytest.mark.parametrize("off_resonance", [True, False])
def test_fp32_inline_phase_paths(M, ctx, oracle_mod, cycles, off_resonance):
    """float32 inline precessions: spin pairs with the packed phase (moderate moments), the
    one-spin float-float path (moments whose products could reach 2^21 cycles) and one spin per
    thread, with and without off-resonance (the Δf·Δt term is skipped when a block has none)."""
    rng = np.random.default_rng(int(cycles) % 1000 + int(off_resonance))
    ph = W.random_phantom(2500, rng)
    if not off_resonance:
        ph.dw[:] = 0.0
    seq = _inline_phase_sequence(rng, cycles)
    ref = oracle_mod.signal(ph, seq)
    for k, t in ((4, 128), (2, 64), (8, 64), (1, 128)):
        out = run(M, ctx, ph, seq, M.FP32, spins_per_thread=k, threads_per_block=t)
        assert rel_l2(out, ref) <= TOL32, (k, t)


@pytest.mark.parametrize("prec,shapes", [
    ("fp32", [(1, 32), (1, 64), (1, 512), (2, 128), (2, 512), (4, 96), (4, 512), (8, 64), (8, 256)]),
    ("fp64", [(1, 32), (1, 256), (2, 64), (2, 256)]),
])
def test_launch_shapes_agree(M, ctx, oracle_mod, prec, shapes):
    rng = np.random.default_rng(77)
    ph = W.random_phantom(3001, rng)
    seq = W.random_sequence(600, rng)
    ref = oracle_mod.signal(ph, seq)
    p = M.FP32 if prec == "fp32" else M.FP64
    tol = TOL32 if prec == "fp32" else TOL64
    tol = max(tol, fp64_phase_tolerance(ph, seq)) if p == M.FP64 else tol
    ran = 0
    for k, t in shapes:
        try:
            out = run(M, ctx, ph, seq, p, spins_per_thread=k, threads_per_block=t)
        except M.MrsimError as e:  # the shape's shared memory exceeds the device limit
            assert e.status == M.Status.EUNSUPPORTED, (k, t, e)
            continue
        assert rel_l2(out, ref) <= tol, (k, t)
        ran += 1
    assert ran >= len(shapes) - 2


def test_state_resume_equals_single_run(M, ctx, oracle_mod):
    """Checkpoint / resume: two consecutive sub-sequences chained through state_out → state_in."""
    w = W.config1()
    ev = w.sequence.events
    cut = 67 * 23 + 30  # inside a readout
    a = W.Sequence(ev[:cut], w.sequence.gamma_hz_per_t)
    b = W.Sequence(ev[cut:], w.sequence.gamma_hz_per_t)
    ref = oracle_mod.signal(w)
    for prec, tol in ((M.FP64, TOL64), (M.FP32, TOL32)):
        st = np.zeros((w.phantom.n, 3))
        sa = run(M, ctx, w.phantom, a, prec, state_out=st)
        sb = run(M, ctx, w.phantom, b, prec, state_in=st)
        assert rel_l2(np.concatenate([sa, sb]), ref) <= tol


def test_accumulate_over_spin_subsets(M, ctx):
    """Domain decomposition (§5.3.2): the signal of the whole object is the sum over subsets."""
    w = W.config1()
    seq = M.Sequence.from_workload_sequence(ctx, w.sequence)
    full = M.simulate(ctx, M.Phantom.from_workload_phantom(ctx, w.phantom), seq, M.FP64)
    idx = np.random.default_rng(3).permutation(w.phantom.n)
    acc = np.zeros(seq.n_adc, dtype=complex)
    for part in np.array_split(idx, 3):
        M.simulate(ctx, M.Phantom.from_workload_phantom(ctx, w.phantom.subset(part)), seq, M.FP64, out=acc, accumulate=True)
    assert rel_l2(acc, full) <= 1e-13


def test_edge_cases(M, ctx, oracle_mod):
    rng = np.random.default_rng(9)
    seq = W.random_sequence(300, rng)
    # zero spins: zero signal
    empty = W.random_phantom(0, rng)
    for p in (M.FP64, M.FP32):
        out = run(M, ctx, empty, seq, p)
        assert out.shape == (seq.n_adc,) and not np.any(out)
    # one spin, T = inf, Δt = 0 events; a sequence without any sample
    one = W.random_phantom(1, rng)
    one.t1[:] = np.inf
    one.t2[:] = np.inf
    ev = np.concatenate([W.make_events([(0.0, 0, 0, 0, 1.0, 0.3, 1, 0.2), (0.0, 1e-3, 0, 0, 0, 0, 1, 0.0)]), seq.events])
    s1 = W.Sequence(ev, W.GAMMA_BAR)
    ref = oracle_mod.signal(one, s1)
    assert rel_l2(run(M, ctx, one, s1, M.FP64), ref) <= TOL64
    assert rel_l2(run(M, ctx, one, s1, M.FP32), ref) <= TOL32
    noadc = W.Sequence(seq.events[seq.events["adc"] == 0], W.GAMMA_BAR)
    st = np.zeros((one.n, 3))
    out = run(M, ctx, one, noadc, M.FP64, state_out=st)
    _, ref_st = oracle_mod.simulate(one, noadc.events, W.GAMMA_BAR, want_signal=False, want_state=True)
    assert out.shape == (0,)
    assert np.max(np.abs(st - ref_st)) <= 1e-12


def test_invalid_inputs(M, ctx):
    rng = np.random.default_rng(10)
    ph = W.random_phantom(10, rng)
    bad = ph.subset(np.arange(10))
    bad.t1[3] = 0.0
    with pytest.raises(M.MrsimError) as e:
        M.Phantom.from_workload_phantom(ctx, bad)
    assert e.value.status == M.Status.EINVAL
    bad = ph.subset(np.arange(10))
    bad.x[7] = np.nan
    with pytest.raises(M.MrsimError):
        M.Phantom.from_workload_phantom(ctx, bad)
    seq = M.Sequence.from_workload_sequence(ctx, W.random_sequence(50, rng))
    p = M.Phantom.from_workload_phantom(ctx, ph)
    out = np.zeros(seq.n_adc + 1, dtype=complex)
    import ctypes

    rc = M.lib().mrsim_simulate(ctx.h, p.h, seq.h, M.FP32, None, ctypes.c_void_p(out.ctypes.data), seq.n_adc + 1)
    assert rc == M.Status.EINVAL
    with pytest.raises(M.MrsimError):
        M.simulate(ctx, p, seq, M.FP32, spins_per_thread=3)


def test_device_buffers_and_streams(M, ctx, oracle_mod):
    torch = pytest.importorskip("torch")
    w = W.config1()
    dev = torch.device("cuda:0")
    arrs = [torch.from_numpy(a).to(dev) for a in w.phantom.arrays()]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = M.Phantom(ctx, arrs, stream=s)
        seq = M.Sequence.from_workload_sequence(ctx, w.sequence)
        out = torch.zeros(2 * seq.n_adc, dtype=torch.float64, device=dev)
        M.simulate(ctx, p, seq, M.FP32, stream=s, out=out)
    s.synchronize()
    ctx.stream_status(s)
    got = out.cpu().numpy().view(np.complex128)
    assert rel_l2(got, oracle_mod.signal(w)) <= TOL32


def test_config2_subset_parity(M, ctx, oracle_mod):
    """Full C2 sequence (sinc 90/180, B0 + fat) on a random subset of its spins."""
    w = W.config2()
    idx = np.sort(np.random.default_rng(21).choice(w.phantom.n, 1500, replace=False))
    sub = w.phantom.subset(idx)
    ref = oracle_mod.signal(sub, w.sequence)
    assert rel_l2(run(M, ctx, sub, w.sequence, M.FP64), ref) <= TOL64
    assert rel_l2(run(M, ctx, sub, w.sequence, M.FP32), ref) <= TOL32


def test_rasterized_sequences_parity(M, ctx, oracle_mod):
    """The 10 µs rasterized stress lists: C1 against the oracle on the rasterized list itself, and
    a C2 spin subset against the oracle on the canonical list (the two lists give the same signal:
    Eq. 4.1 composes over the pieces, pinned on the CPU)."""
    w = W.config1()
    r = W.rasterize(w.sequence)
    ref = oracle_mod.signal(w.phantom, r)
    # the oracle turns every spin once per event: each turn's cos/sin rounding changes |M| by up to
    # about 2^-52, so on 64 000 events its own float64 floor is 2·2^-53·n_events ≈ 1.4e-11
    # (the library merges the pieces and turns once per canonical interval)
    tol64 = max(TOL64, 2 * 2.0**-53 * r.n_events)
    assert rel_l2(run(M, ctx, w.phantom, r, M.FP64), ref) <= tol64
    assert rel_l2(run(M, ctx, w.phantom, r, M.FP32), ref) <= TOL32
    w = W.config2()
    sub = w.phantom.subset(np.sort(np.random.default_rng(22).choice(w.phantom.n, 1200, replace=False)))
    ref = oracle_mod.signal(sub, w.sequence)
    r = W.rasterize(w.sequence)
    assert rel_l2(run(M, ctx, sub, r, M.FP64), ref) <= TOL64
    assert rel_l2(run(M, ctx, sub, r, M.FP32), ref) <= TOL32


def test_config2_full_size_fp32_vs_fp64(M, ctx):
    """Full-size C2 in the benchmark's launch shape: float32 against the float64 GPU path, and
    additivity of the float64 path over two disjoint halves of the spins."""
    w = W.config2()
    seq = M.Sequence.from_workload_sequence(ctx, w.sequence)
    p = M.Phantom.from_workload_phantom(ctx, w.phantom)
    s64 = M.simulate(ctx, p, seq, M.FP64)
    s32 = M.simulate(ctx, p, seq, M.FP32)
    assert rel_l2(s32, s64) <= TOL32
    half = w.phantom.n // 2
    acc = np.zeros(seq.n_adc, dtype=complex)
    for part in (np.arange(half), np.arange(half, w.phantom.n)):
        M.simulate(ctx, M.Phantom.from_workload_phantom(ctx, w.phantom.subset(part)), seq, M.FP64, out=acc, accumulate=True)
    assert rel_l2(acc, s64) <= 1e-13


def test_config3_subset_parity(M, ctx, oracle_mod):
    """Full C3 sequence (3D RF-spoiled GRE, 2.1 M events) on a random subset of its spins."""
    w = W.config3()
    idx = np.sort(np.random.default_rng(31).choice(w.phantom.n, 384, replace=False))
    sub = w.phantom.subset(idx)
    ref = oracle_mod.signal(sub, w.sequence)
    assert rel_l2(run(M, ctx, sub, w.sequence, M.FP64), ref) <= TOL64
    assert rel_l2(run(M, ctx, sub, w.sequence, M.FP32), ref) <= TOL32


def test_sequence_from_host_compiled_program(M, ctx, oracle_mod):
    """mrsim_compile on a worker thread + mrsim_sequence_create equals mrsim_sequence_load; the
    sequence keeps the program's tables after the compiled handle is destroyed."""
    from concurrent.futures import ThreadPoolExecutor

    w = W.config1()
    with ThreadPoolExecutor(1) as pool:
        comp = pool.submit(M.Compiled, w.sequence.events, w.sequence.gamma_hz_per_t).result()
    s = M.Sequence.from_compiled(ctx, comp)
    comp.close()
    assert s.n_adc == w.sequence.n_adc and s.n_events == w.sequence.n_events
    p = M.Phantom.from_workload_phantom(ctx, w.phantom)
    ref = oracle_mod.signal(w)
    plain = M.Sequence.from_workload_sequence(ctx, w.sequence)
    for prec, tol in ((M.FP64, TOL64), (M.FP32, TOL32)):
        got = M.simulate(ctx, p, s, prec)
        assert rel_l2(got, ref) <= tol
        assert rel_l2(got, M.simulate(ctx, p, plain, prec)) <= tol
    s.close()
    plain.close()
    p.close()


def test_bounded_wait_timeout_is_reported(M, ctx, oracle_mod):
    """Failure detection without a fault: the kernels' bounded mbarrier wait, run on a barrier that
    nothing completes with a 20 ms limit, gives up, records MRSIM_ETIMEOUT in the status word,
    which the next status read reports and clears; the context keeps working."""
    L = M.lib()
    assert L.mrsim_debug_wait_timeout(ctx.h, 20_000_000, None) == 0
    assert L.mrsim_stream_status(ctx.h, None) == 4  # MRSIM_ETIMEOUT
    assert L.mrsim_stream_status(ctx.h, None) == 0  # cleared
    assert L.mrsim_debug_wait_timeout(ctx.h, 10, None) == 1  # limit outside [1e3, 1e9] ns
    w = W.config1()
    ref = oracle_mod.signal(w)
    assert rel_l2(run(M, ctx, w.phantom, w.sequence, M.FP64), ref) <= TOL64


@pytest.mark.parametrize("what", ["phantom", "sequence", "host_output"])
def test_allocation_failure_is_reported(M, oracle_mod, what):
    """Out-of-memory without exhausting the device: the failure hook makes the next device
    allocation of the call fail; the call returns MRSIM_ENOMEM, leaves nothing half-built and the
    same call succeeds afterwards (the hook fires once)."""
    w = W.config1()
    L = M.lib()
    c = M.Context(0)  # fresh: its host-output scratch is not allocated yet
    try:
        p = M.Phantom.from_workload_phantom(c, w.phantom) if what != "phantom" else None
        s = M.Sequence.from_workload_sequence(c, w.sequence) if what == "host_output" else None
        assert L.mrsim_debug_fail_alloc(c.h, 0) == 0
        with pytest.raises(M.MrsimError) as e:
            if what == "phantom":
                M.Phantom.from_workload_phantom(c, w.phantom)
            elif what == "sequence":
                M.Sequence.from_workload_sequence(c, w.sequence)
            else:
                M.simulate(c, p, s, M.FP64)
        assert e.value.status == M.Status.ENOMEM
        if p is None:
            p = M.Phantom.from_workload_phantom(c, w.phantom)
        if s is None:
            s = M.Sequence.from_workload_sequence(c, w.sequence)
        assert rel_l2(M.simulate(c, p, s, M.FP64), oracle_mod.signal(w)) <= TOL64
        c.stream_status()
        p.close()
        s.close()
    finally:
        c.close()


def test_autotune_cache_file(M, tmp_path):
    """MRSIM_AUTOTUNE_CACHE: the first process tunes and appends its shape; a second process
    loads it and answers mrsim_autotune without timing (same shape, no new line)."""
    import subprocess
    import sys

    cache = tmp_path / "tune.txt"
    code = ("import time, numpy as np\n"
            "from paper_1305_6861_gb300 import mrsim as M, workloads as W\n"
            "w = W.config2(n=64, iso=2)\nctx = M.Context(0)\n"
            "p = M.Phantom.from_workload_phantom(ctx, w.phantom)\ns = M.Sequence.from_workload_sequence(ctx, w.sequence)\n"
            "t0 = time.perf_counter(); k, t = M.autotune(ctx, p, s, M.FP32); dt = time.perf_counter() - t0\n"
            "print(k, t, dt)\n")
    env = dict(os.environ, MRSIM_AUTOTUNE_CACHE=str(cache))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(r.stdout.split())
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("mrsim-tune-1 ")
    assert outs[0][:2] == outs[1][:2]
    assert float(outs[1][2]) < float(outs[0][2])


def test_allocation_failure_from_environment(M):
    """MRSIM_FAIL_ALLOC arms the allocation-failure hook in a process that does not call the
    library's hook itself: its first phantom upload fails with ENOMEM, the second succeeds."""
    import subprocess
    import sys

    code = ("from paper_1305_6861_gb300 import mrsim as M, workloads as W\n"
            "w = W.config1()\nctx = M.Context(0)\n"
            "try:\n    M.Phantom.from_workload_phantom(ctx, w.phantom)\n    print('no failure')\n"
            "except M.MrsimError as e:\n    print(e.status.name)\n"
            "p = M.Phantom.from_workload_phantom(ctx, w.phantom)\nprint('ok', p.n)\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=dict(os.environ, MRSIM_FAIL_ALLOC="0"),
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.split() == ["ENOMEM", "ok", "4096"], r.stdout


def test_rasterized_snapshots_parity(M, ctx, oracle_mod):
    """Snapshots in the middle of split intervals of a rasterized list (the compiler ends the
    merge there) in both precisions against the oracle's prefix states."""
    rng = np.random.default_rng(78)
    ph = W.random_phantom(1500 + 37, rng)
    w = W.config1()
    seq = W.rasterize(W.Sequence(w.sequence.events[: 67 * 4], w.sequence.gamma_hz_per_t), 2.5e-6)
    ev = seq.events
    mid = np.nonzero((ev["adc"] == 0) & (ev["rf_flip"] == 0))[0]
    snaps = np.sort(rng.choice(mid, size=4, replace=False))
    p = M.Phantom.from_workload_phantom(ctx, ph)
    s = M.Sequence(ctx, ev, seq.gamma_hz_per_t, snapshots=snaps)
    ref_sig, _ = oracle_mod.simulate(ph, ev, seq.gamma_hz_per_t)
    refs = [oracle_mod.simulate(ph, ev[: e + 1], seq.gamma_hz_per_t, want_signal=False, want_state=True)[1]
            for e in snaps]
    tol64 = max(TOL64, 2 * 2.0**-53 * len(ev))
    for prec, tol_s, tol_m in ((M.FP64, tol64, tol64), (M.FP32, TOL32, 1e-4)):
        out = np.zeros((len(snaps), ph.n, 3))
        sig = M.simulate(ctx, p, s, prec, snapshots=out)
        ctx.stream_status()
        assert rel_l2(sig, ref_sig) <= tol_s
        for q in range(len(snaps)):
            assert np.max(np.abs(out[q] - refs[q])) <= tol_m, (prec, q)


def test_compensated_precision(M, ctx, oracle_mod):
    """MRSIM_FP32_KAHAN: the forward path in double-float arithmetic on the FP32 pipe (every
    product and sum carries its rounding error, about 48 significant bits).  Against the float64
    oracle at 1e-10 (a derived bar: ~2^-44 relative per compensated operation, summed in
    quadrature over the ~1e5 operations a spin sees) on C1 and on random sequences in several
    launch shapes with a ragged tail, state out included; the calls without a compensated kernel
    (receive coils) serve it with float32; an unknown precision is refused."""
    import ctypes

    TOLK = 1e-10
    w = W.config1()
    ref = oracle_mod.signal(w)
    p = M.Phantom.from_workload_phantom(ctx, w.phantom)
    s = M.Sequence.from_workload_sequence(ctx, w.sequence)
    got = M.simulate(ctx, p, s, M.FP32_KAHAN)
    assert rel_l2(got, ref) <= TOLK
    rng = np.random.default_rng(4321)
    ph = W.random_phantom(1777, rng)
    ph.dw[:] = 2 * math.pi * rng.uniform(-80, 80, ph.n)
    seq = W.random_sequence(800, rng, runs=True)
    r2, rst = oracle_mod.simulate(ph, seq.events, seq.gamma_hz_per_t, want_state=True)
    tol = max(TOLK, fp64_phase_tolerance(ph, seq))
    for k, t in ((1, 32), (1, 256), (2, 64), (2, 256)):
        st = np.zeros((ph.n, 3))
        g = run(M, ctx, ph, seq, M.FP32_KAHAN, spins_per_thread=k, threads_per_block=t, state_out=st)
        assert rel_l2(g, r2) <= tol, (k, t, rel_l2(g, r2))
        assert np.max(np.abs(st - rst)) <= tol * max(1.0, np.abs(rst).max())
    sens = np.ones((2, w.phantom.n), dtype=complex)
    ca = M.simulate_coils(ctx, p, s, sens, M.FP32)
    cb = M.simulate_coils(ctx, p, s, sens, M.FP32_KAHAN)
    assert rel_l2(cb, ca) <= 1e-6
    out = np.zeros(s.n_adc, dtype=complex)
    rc = M.lib().mrsim_simulate(ctx.h, p.h, s.h, 3, None, ctypes.c_void_p(out.ctypes.data), s.n_adc)
    assert rc == M.Status.EINVAL


def test_compensated_precision_on_c2_and_autotune(M, ctx, oracle_mod):
    """The compensated precision on the C2 spin echo (sub-pulse trains, B0 + fat) on a spin subset
    against the oracle, and its autotuned shape (a float64-style shape)."""
    w = W.config2()
    sub = w.phantom.subset(np.sort(np.random.default_rng(24).choice(w.phantom.n, 1500, replace=False)))
    ref = oracle_mod.signal(sub, w.sequence)
    p = M.Phantom.from_workload_phantom(ctx, sub)
    s = M.Sequence.from_workload_sequence(ctx, w.sequence)
    k, t = M.autotune(ctx, p, s, M.FP32_KAHAN)
    assert k in (1, 2) and 32 <= t <= 256
    assert rel_l2(M.simulate(ctx, p, s, M.FP32_KAHAN), ref) <= 1e-10


def test_config2_legendre_field_parity(M, ctx, oracle_mod):
    """C2 with the Eq. 6.3 inhomogeneity (C = 20 µT, homogeneity sphere of diameter 0.5 m) on spin
    subsets, both precisions: spins inside 0.9 R (offsets up to a few hundred Hz) at the 1e-12 /
    2e-5 bars; spins anywhere in the 0.5 m field of view (up to 12.7 kHz at the corners, phases of
    ~4e4 rad per rest interval) at the float64 floor those phases set and the float32 bar."""
    w = W.config2_legendre()
    ph = w.phantom
    r = np.sqrt(ph.x**2 + ph.y**2 + ph.z**2)
    rng = np.random.default_rng(23)
    inner = np.sort(rng.choice(np.nonzero((r < 0.9 * 0.25) & (ph.rho > 0))[0], 1200, replace=False))
    anywhere = np.sort(rng.choice(ph.n, 1200, replace=False))
    for idx, tol64 in ((inner, TOL64), (anywhere, None)):
        sub = ph.subset(idx)
        ref = oracle_mod.signal(sub, w.sequence)
        t64 = tol64 if tol64 is not None else fp64_phase_tolerance(sub, w.sequence)
        assert rel_l2(run(M, ctx, sub, w.sequence, M.FP64), ref) <= t64
        assert rel_l2(run(M, ctx, sub, w.sequence, M.FP32), ref) <= TOL32
