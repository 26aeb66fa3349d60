"""The 3D 128³ RF-spoiled gradient echo (4 194 304 spins, 2 146 304 events, 2 097 152 samples) at
full size, in the launch shape the benchmark times.

* The oracle on a seeded sample of the tissue spins (0.1 % of all spins, several full thread
  blocks' worth) against the GPU: float32 from a launch of the WHOLE phantom with M0 = 0 outside
  the sample (such a spin stays at (0, 0, 0) through every event and adds exact zeros), so the
  sample's spins run in the benchmark's own blocks, next to zeroed neighbours, through its
  cross-block float64 sums; float64 from the sample alone.
* The full float32 signal against the full float64 GPU signal (relative L2 <= 2e-5).
"""
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
def c3(M, ctx):
    w = W.config3()
    seq = M.Sequence.from_workload_sequence(ctx, w.sequence)
    p = M.Phantom.from_workload_phantom(ctx, w.phantom)
    shape = M.autotune(ctx, p, seq, M.FP32)  # the benchmark tunes the same way
    yield w, seq, p, shape
    p.close()
    seq.close()


def masked(ph, idx):
    rho = np.zeros_like(ph.rho)
    rho[idx] = ph.rho[idx]
    return W.Phantom(ph.x, ph.y, ph.z, rho, ph.t1, ph.t2, ph.dw)


def test_config3_oracle_sample_through_the_bench_launch(M, ctx, oracle_mod, c3):
    w, seq, _, shape = c3
    tissue = np.nonzero(w.phantom.rho > 0)[0]
    m = int(round(1e-3 * w.phantom.n))  # 4 194 spins
    idx = np.sort(np.random.default_rng(31).choice(tissue, m, replace=False))
    ref = oracle_mod.signal(w.phantom.subset(idx), w.sequence)
    assert np.linalg.norm(ref) > 0
    pm = M.Phantom.from_workload_phantom(ctx, masked(w.phantom, idx))
    shapes = [tuple(shape)] + [s for s in ((4, 256), (8, 224), (2, 256)) if s != tuple(shape)]
    ran = 0
    for k, t in shapes:
        try:
            got = M.simulate(ctx, pm, seq, M.FP32, spins_per_thread=k, threads_per_block=t)
        except M.MrsimError as e:  # a shape whose shared memory exceeds the device limit
            assert e.status == M.Status.EUNSUPPORTED and (k, t) != tuple(shape), (k, t, e)
            continue
        ctx.stream_status()
        assert rel_l2(got, ref) <= TOL32, (k, t)
        ran += 1
    assert ran >= 2
    pm.close()
    ps = M.Phantom.from_workload_phantom(ctx, w.phantom.subset(idx))
    assert rel_l2(M.simulate(ctx, ps, seq, M.FP64), ref) <= TOL64
    ps.close()


def test_config3_full_signal_fp32_vs_fp64(M, ctx, c3):
    w, seq, p, (k, t) = c3
    s32 = M.simulate(ctx, p, seq, M.FP32, spins_per_thread=k, threads_per_block=t)
    s64 = M.simulate(ctx, p, seq, M.FP64)
    ctx.stream_status()
    assert s32.shape == (2_097_152,)
    assert rel_l2(s32, s64) <= TOL32
