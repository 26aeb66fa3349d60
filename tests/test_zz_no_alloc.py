"""The batch entry point that allocates nothing (mrsim_simulate_batch_static), for callers that
cannot call cudaMalloc when they simulate (a plug-in whose host application owns every device
allocation, a real-time loop under a fixed memory budget): its output must equal the regular batch
API's and the float64 CPU oracle's, call after call, a call after the first must leave the
device's free memory unchanged, and batches beyond its fixed scratch must be refused with EINVAL.

Kept in a file of its own, collected last, so that a run stopping at the first failure has
already run every other test."""
import ctypes
import math

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def _pairs():
    rng = np.random.default_rng(42)
    out = []
    for i, n in enumerate([3000, 1, 777, 0, 5000]):
        ph = W.random_phantom(n, rng)
        ph.dw[:] = 2 * math.pi * rng.uniform(-50, 50, n)
        if i % 2:
            seq = W.spin_echo(16, 8, 0.5, 12e-3, 30e-3, 10e-6, n_rf=24)
        else:
            seq = W.flash(16, 16, 0.5, 0.4, 5e-3, 2.5e-3, 10e-6, rf_spoil=bool(i % 4))
        out.append((ph, seq))
    return out


@pytest.mark.parametrize("prec,tol,tol_oracle", [("fp32", 1e-6, 2e-5), ("fp64", 1e-12, 1e-12),
                                                 ("fp32_kahan", 1e-12, 1e-10)])
def test_static_scratch_batch_matches_batch_api(mrsim_lib, oracle_mod, prec, tol, tol_oracle):
    torch = pytest.importorskip("torch")
    M = mrsim_lib
    p = {"fp32": M.FP32, "fp64": M.FP64, "fp32_kahan": M.FP32_KAHAN}[prec]
    ctx = M.Context(0)
    # the static call has no memory for train maps and runs every shaped pulse sub-pulse by
    # sub-pulse; the reference batch does the same, so the two compare like for like
    ctx.set_train_maps(False)
    pairs = _pairs()
    oracle_refs = [oracle_mod.signal(ph, seq) for ph, seq in pairs]
    phs = [M.Phantom.from_workload_phantom(ctx, a) for a, _ in pairs]
    sqs = [M.Sequence.from_workload_sequence(ctx, s) for _, s in pairs]
    ref_out = [torch.zeros(max(2 * q.n_adc, 2), dtype=torch.float64, device="cuda") for q in sqs]
    b = M.Batch(ctx, phs, sqs, p, ref_out)
    b.set_shape(2, 64)
    b.launch()
    torch.cuda.synchronize()
    ctx.stream_status()
    ref = [o.cpu().numpy()[: 2 * q.n_adc].view(np.complex128) for o, q in zip(ref_out, sqs)]
    out = [torch.full((max(2 * q.n_adc, 2),), 7.0, dtype=torch.float64, device="cuda") for q in sqs]
    for call in range(2):  # two calls in a row share the static scratch
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        M.simulate_batch_static(ctx, phs, sqs, p, out, spins_per_thread=2, threads_per_block=64)
        torch.cuda.synchronize()
        if call:  # the first call may load the module; later ones take no device memory at all
            assert torch.cuda.mem_get_info()[0] == free_before
        ctx.stream_status()
        got = [o.cpu().numpy()[: 2 * q.n_adc].view(np.complex128) for o, q in zip(out, sqs)]
        for i, (g, r, o) in enumerate(zip(got, ref, oracle_refs)):
            assert rel_l2(g, r) <= tol, (call, i)
            assert rel_l2(g, o) <= tol_oracle, (call, i)
    b.close()
    ctx.close()


def test_static_scratch_limits(mrsim_lib):
    torch = pytest.importorskip("torch")
    M = mrsim_lib
    ctx = M.Context(0)
    seq = M.Sequence.from_workload_sequence(ctx, W.flash(8, 8, 0.5, 0.3, 5e-3, 2.5e-3, 10e-6))
    ph = M.Phantom.from_workload_phantom(ctx, W.random_phantom(4, np.random.default_rng(1)))
    n = 20000  # more descriptors than the 1 MiB scratch holds
    outs = [torch.zeros(2 * seq.n_adc, dtype=torch.float64, device="cuda")]
    arr_p = (ctypes.c_void_p * n)(*([ph.h.value] * n))
    arr_s = (ctypes.c_void_p * n)(*([seq.h.value] * n))
    arr_o = (ctypes.c_void_p * n)(*([outs[0].data_ptr()] * n))
    rc = M.lib().mrsim_simulate_batch_static(ctx.h, n, arr_p, arr_s, M.FP32, None, arr_o, 1, 32)
    assert rc == M.Status.EINVAL
    assert b"static scratch" in M.lib().mrsim_last_error(ctx.h)
    ctx.close()


def test_static_scratch_library_shape_and_current_device(mrsim_lib, oracle_mod):
    """With the library's default shape (0, 0) the call serves the same batch as the batch API
    and gives the caller's current device back unchanged."""
    torch = pytest.importorskip("torch")
    M = mrsim_lib
    ctx = M.Context(0)
    pairs = _pairs()
    phs = [M.Phantom.from_workload_phantom(ctx, a) for a, _ in pairs]
    sqs = [M.Sequence.from_workload_sequence(ctx, s) for _, s in pairs]
    out = [torch.zeros(max(2 * q.n_adc, 2), dtype=torch.float64, device="cuda") for q in sqs]
    dev_before = torch.cuda.current_device()
    M.simulate_batch_static(ctx, phs, sqs, M.FP32, out)
    assert torch.cuda.current_device() == dev_before
    torch.cuda.synchronize()
    ctx.stream_status()
    for (ph, seq), o, q in zip(pairs, out, sqs):
        g = o.cpu().numpy()[: 2 * q.n_adc].view(np.complex128)
        assert rel_l2(g, oracle_mod.signal(ph, seq)) <= 2e-5
    with pytest.raises(ValueError):
        M.simulate_batch_static(ctx, phs, sqs[:-1], M.FP32, out)
    ctx.close()
