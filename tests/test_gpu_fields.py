"""Non-parallel fields on the GPU (mrsim_simulate_fields, §3.2 and §3.4.3.2) against the oracle:
per-spin static-field directions (small tilts and arbitrary directions), gradient fields with
transverse components, low and high main field, several thread blocks with a ragged tail, both
precisions (relative L2 of the signal: float64 at the phase-rounding floor of the sequence, at
least 1e-12; float32 2e-5); the parallel case equals the standard path; invalid inputs."""
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


def directions(rng, n, max_tilt):
    ct = rng.uniform(math.cos(max_tilt), 1.0, n)
    st = np.sqrt(1 - ct**2)
    ph = rng.uniform(0, 2 * math.pi, n)
    return np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)


def case(rng, n_spins, n_events, transverse=True):
    ph = W.random_phantom(n_spins, rng)
    ph.dw[:] = 2 * math.pi * rng.uniform(-100, 100, n_spins)
    rows = []
    for _ in range(n_events):
        flip = rng.uniform(-math.pi, math.pi) if rng.uniform() < 0.1 else 0.0
        g = rng.uniform(-5e-3, 5e-3, 3) if rng.uniform() < 0.8 else np.zeros(3)
        dt = rng.uniform(0.0, 3e-4) if rng.uniform() < 0.95 else 0.0
        rows.append((dt, *g, flip, rng.uniform(0, 2 * math.pi), int(rng.uniform() < 0.4), rng.uniform(0, 2 * math.pi)))
    ev = W.make_events(rows)
    gt = None
    if transverse:
        gt = rng.uniform(-4e-3, 4e-3, (n_events, 6))
        gt[rng.uniform(size=n_events) < 0.4] = 0.0
    return ph, ev, gt


def phase_floor(ph, ev, gt, b0):
    """float64 floor of a sequence: each side rounds every event's angle with relative error
    2^-53, so 4 * 2^-53 * sqrt(sum of squared angles) bounds the relative signal difference."""
    x = np.stack([ph.x, ph.y, ph.z], axis=1)
    g = np.stack([ev["gx"], ev["gy"], ev["gz"]], axis=1)
    b = np.abs(g) @ np.abs(x).max(axis=0)
    if gt is not None:
        b = b + np.abs(gt[:, :3]) @ np.abs(x).max(axis=0) + np.abs(gt[:, 3:]) @ np.abs(x).max(axis=0)
    th = (2 * math.pi * W.GAMMA_BAR * b + np.abs(ph.dw).max()) * ev["dt"]
    return max(TOL64, 4 * 2.0**-53 * float(np.sqrt(np.sum(th**2))))


@pytest.mark.parametrize("seed,n_spins,n_events,max_tilt,b0,transverse", [
    (0, 3001, 700, 0.2, 1.5, True),       # small tilts, transverse gradients, 1.5 T
    (1, 1000, 500, math.pi, 0.05, True),  # arbitrary directions at a low main field
    (2, 257, 900, 1.0, 0.3, False),       # tilted fields, parallel gradients only
    (3, 1, 300, math.pi, 1.0, True),      # one spin
])
def test_fields_match_oracle(M, ctx, oracle_mod, seed, n_spins, n_events, max_tilt, b0, transverse):
    rng = np.random.default_rng(900 + seed)
    ph, ev, gt = case(rng, n_spins, n_events, transverse)
    nd = directions(rng, n_spins, max_tilt)
    ref, _ = oracle_mod.simulate_fields(ph, ev, W.GAMMA_BAR, nd, gt, b0)
    p = M.Phantom.from_workload_phantom(ctx, ph)
    M.set_b0_direction(ctx, p, nd)
    f = M.Fields(ctx, ev, W.GAMMA_BAR, gt, b0)
    got64 = M.simulate_fields(ctx, p, f, M.FP64)
    got32 = M.simulate_fields(ctx, p, f, M.FP32)
    ctx.stream_status()
    assert rel_l2(got64, ref) <= phase_floor(ph, ev, gt, b0)
    assert rel_l2(got32, ref) <= TOL32


def test_fields_parallel_case_is_the_standard_path(M, ctx, oracle_mod):
    """n = z everywhere and no transverse components: the C1 FLASH through the field path equals the
    oracle (1e-12 / 2e-5) and the standard path."""
    w = W.config1()
    ev = w.sequence.events
    nd = np.tile([0.0, 0.0, 1.0], (w.phantom.n, 1))
    ref = oracle_mod.signal(w)
    p = M.Phantom.from_workload_phantom(ctx, w.phantom)
    s = M.Sequence.from_workload_sequence(ctx, w.sequence)
    std = M.simulate(ctx, p, s, M.FP64)
    got64 = M.simulate_fields(ctx, p, M.Fields(ctx, ev, W.GAMMA_BAR, None, 1.5), M.FP64)  # no directions: z
    M.set_b0_direction(ctx, p, nd)
    got32 = M.simulate_fields(ctx, p, M.Fields(ctx, ev, W.GAMMA_BAR, np.zeros((len(ev), 6)), 1.5), M.FP32)
    assert rel_l2(got64, ref) <= TOL64 and rel_l2(got64, std) <= TOL64
    assert rel_l2(got32, ref) <= TOL32


def test_fields_device_buffers(M, ctx, oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(905)
    ph, ev, gt = case(rng, 700, 400)
    nd = directions(rng, ph.n, 0.5)
    ref, _ = oracle_mod.simulate_fields(ph, ev, W.GAMMA_BAR, nd, gt, 0.5)
    p = M.Phantom.from_workload_phantom(ctx, ph)
    dev = torch.device("cuda:0")
    ndd = torch.from_numpy(nd.reshape(-1).copy()).to(dev)
    M.set_b0_direction(ctx, p, ndd)
    f = M.Fields(ctx, ev, W.GAMMA_BAR, gt, 0.5)
    out = torch.zeros(2 * f.n_adc, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream()
    M.simulate_fields(ctx, p, f, M.FP64, stream=s, out=out)  # asynchronous on s
    s.synchronize()
    ctx.stream_status(s)
    assert rel_l2(out.cpu().numpy().view(np.complex128), ref) <= phase_floor(ph, ev, gt, 0.5)


def test_fields_edge_cases_and_invalid_inputs(M, ctx, oracle_mod):
    rng = np.random.default_rng(906)
    ph, ev, gt = case(rng, 50, 100)
    nd = directions(rng, ph.n, 1.0)
    p = M.Phantom.from_workload_phantom(ctx, ph)
    M.set_b0_direction(ctx, p, nd)
    f = M.Fields(ctx, ev, W.GAMMA_BAR, gt, 1.5)
    # no spins: zero signal; no events: empty signal
    p0 = M.Phantom.from_workload_phantom(ctx, W.random_phantom(0, rng))
    M.set_b0_direction(ctx, p0, np.zeros((0, 3)))
    f0 = M.Fields(ctx, ev[:0], W.GAMMA_BAR, None, 1.5)
    for prec in (M.FP64, M.FP32):
        z = M.simulate_fields(ctx, p0, f, prec)
        assert z.shape == (f.n_adc,) and not np.any(z)
        assert M.simulate_fields(ctx, p, f0, prec).shape == (0,)
    bad = nd.copy()
    bad[7] *= 1.01  # not a unit vector
    with pytest.raises(M.MrsimError) as e:
        M.set_b0_direction(ctx, p, bad)
    assert e.value.status == M.Status.EINVAL and "spin 7" in str(e.value)
    for b0 in (0.0, -1.0, float("nan")):
        with pytest.raises(M.MrsimError) as e:
            M.Fields(ctx, ev, W.GAMMA_BAR, gt, b0)
        assert e.value.status == M.Status.EINVAL
    g_bad = gt.copy()
    g_bad[3, 2] = np.inf
    with pytest.raises(M.MrsimError):
        M.Fields(ctx, ev, W.GAMMA_BAR, g_bad, 1.5)
    out = np.zeros(f.n_adc + 1, dtype=complex)
    import ctypes

    rc = M.lib().mrsim_simulate_fields(ctx.h, p.h, f.h, M.FP64, None, ctypes.c_void_p(out.ctypes.data), f.n_adc + 1)
    assert rc == M.Status.EINVAL
    # the failed direction update kept the earlier directions; the context stays usable
    ref, _ = oracle_mod.simulate_fields(ph, ev, W.GAMMA_BAR, nd, gt, 1.5)
    assert rel_l2(M.simulate_fields(ctx, p, f, M.FP64), ref) <= phase_floor(ph, ev, gt, 1.5)


def test_fields_workload_c1_low_field(M, ctx, oracle_mod):
    """The 64² FLASH at 0.05 T with a 10° smooth tilt and Maxwell concomitant fields, every spin,
    both precisions."""
    w = W.config_fields()
    ref, _ = oracle_mod.simulate_fields(w.phantom, w.sequence.events, W.GAMMA_BAR, w.b0_dir, w.g_transverse,
                                        w.b0_tesla)
    p = M.Phantom.from_workload_phantom(ctx, w.phantom)
    M.set_b0_direction(ctx, p, w.b0_dir)
    f = M.Fields(ctx, w.sequence.events, W.GAMMA_BAR, w.g_transverse, w.b0_tesla)
    assert rel_l2(M.simulate_fields(ctx, p, f, M.FP64), ref) <= TOL64
    assert rel_l2(M.simulate_fields(ctx, p, f, M.FP32), ref) <= TOL32


@pytest.mark.parametrize("n_spins", [262143, 60000])
def test_fields_large_launch_masked(M, ctx, oracle_mod, n_spins):
    """A launch of C2's spin count less one (1 024 blocks of the float32 kernel, more than one wave
    of resident blocks, a ragged last block) and a one-wave launch: every spin outside a 240-spin
    sample has M0 = 0 (such a spin stays at zero), so the signal is the sample's, against the
    oracle on the sample; the sample includes the last spins of the phantom."""
    rng = np.random.default_rng(920 + n_spins % 97)
    ph, ev, gt = case(rng, n_spins, 300)
    nd = directions(rng, n_spins, 0.4)
    idx = np.sort(np.concatenate([rng.choice(n_spins - 64, 200, replace=False), np.arange(n_spins - 40, n_spins)]))
    rho = np.zeros_like(ph.rho)
    rho[idx] = ph.rho[idx]
    masked = W.Phantom(ph.x, ph.y, ph.z, rho, ph.t1, ph.t2, ph.dw)
    sub = ph.subset(idx)
    ref, _ = oracle_mod.simulate_fields(sub, ev, W.GAMMA_BAR, nd[idx], gt, 1.0)
    p = M.Phantom.from_workload_phantom(ctx, masked)
    M.set_b0_direction(ctx, p, nd)
    f = M.Fields(ctx, ev, W.GAMMA_BAR, gt, 1.0)
    got32 = M.simulate_fields(ctx, p, f, M.FP32)
    got64 = M.simulate_fields(ctx, p, f, M.FP64)
    ctx.stream_status()
    assert rel_l2(got32, ref) <= TOL32
    assert rel_l2(got64, ref) <= phase_floor(sub, ev, gt, 1.0)


def test_fields_train_maps(M, ctx, oracle_mod):
    """A spin echo whose sinc pulses recur every TR, with tilted static fields and Maxwell
    concomitant components: its trains run as maps (pulse, then the interval's turn, composed per
    spin at set-up) when the context's maps are on at creation, event by event when off; both
    against the oracle at the usual bars."""
    rng = np.random.default_rng(930)
    seq = W.spin_echo(16, 8, 0.5, 12e-3, 30e-3, 10e-6, n_rf=24)
    ev = seq.events
    gt = W.concomitant_transverse(ev)
    ph = W.random_phantom(2001, rng)
    ph.dw[:] = 2 * math.pi * rng.uniform(-80, 80, ph.n)
    nd = directions(rng, ph.n, 0.3)
    ref, _ = oracle_mod.simulate_fields(ph, ev, W.GAMMA_BAR, nd, gt, 0.3)
    p = M.Phantom.from_workload_phantom(ctx, ph)
    M.set_b0_direction(ctx, p, nd)
    floor = phase_floor(ph, ev, gt, 0.3)
    try:
        for maps in (True, False):
            ctx.set_train_maps(maps)
            f = M.Fields(ctx, ev, W.GAMMA_BAR, gt, 0.3)
            assert (f.n_train_maps > 0) == maps
            if maps:  # the benchmark's work model marks the same map kinds as the library
                import bench

                assert f.n_train_maps == len(bench.field_train_maps(ev, gt)[1])
            got64 = M.simulate_fields(ctx, p, f, M.FP64)
            got32 = M.simulate_fields(ctx, p, f, M.FP32)
            ctx.stream_status()
            assert rel_l2(got64, ref) <= floor, (maps, rel_l2(got64, ref))
            assert rel_l2(got32, ref) <= TOL32, (maps, rel_l2(got32, ref))
    finally:
        ctx.set_train_maps(True)

