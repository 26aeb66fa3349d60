"""Rewound readouts on the GPU (the compiler folds phase encoding A and rewinder B into the run:
the run applies A inline before its samples and its anchor restores from the state before A with
the phasor of A+R+B).  Parity with the oracle through the C-ABI in both precisions, with receive
coils, with snapshots that break the fold, and for the overlapping multi-echo case.
Tolerances: float64 the phase floor of the sequence (at least 1e-12), float32 2e-5 rel-L2 on the
signal and 1e-4 on states of magnitude ≤ 1."""
import numpy as np
import pytest

import rewound_cases as RC

pytestmark = pytest.mark.gpu

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


CASES = {
    "fold": lambda: RC.flash_like(n_tr=40, n_read=64),
    "multi_echo": lambda: RC.multi_echo(n_tr=30, n_read=48),
    "missed_rewinder": lambda: RC.flash_like(n_tr=40, n_read=64, jitter=np.random.default_rng(5)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_rewound_parity(M, ctx, oracle_mod, case):
    ev = CASES[case]()
    ph = RC.phantom(3000 + 77, np.random.default_rng(21))  # several blocks and a ragged tail
    ref, ref_state = oracle_mod.simulate(ph, ev, RC.GAMMA, want_state=True)
    p = M.Phantom.from_workload_phantom(ctx, ph)
    s = M.Sequence(ctx, ev, RC.GAMMA)
    tol64 = RC.phase_floor(ph, ev)
    for prec in (M.FP64, M.FP32):
        st = np.zeros((ph.n, 3))
        sig = M.simulate(ctx, p, s, prec, state_out=st)
        ctx.stream_status()
        if prec == M.FP64:
            assert rel_l2(sig, ref) <= tol64
            assert np.max(np.abs(st - ref_state)) <= tol64 * max(1.0, np.abs(ref_state).max())
        else:
            assert rel_l2(sig, ref) <= TOL32
            assert np.max(np.abs(st - ref_state)) <= 1e-4


def test_rewound_coils_parity(M, ctx, oracle_mod):
    ev = RC.flash_like(n_tr=24, n_read=48)
    rng = np.random.default_rng(22)
    ph = RC.phantom(1500 + 33, rng)
    sens = rng.normal(size=(3, ph.n)) + 1j * rng.normal(size=(3, ph.n))
    ref = oracle_mod.simulate_coils(ph, ev, RC.GAMMA, sens)
    p = M.Phantom.from_workload_phantom(ctx, ph)
    s = M.Sequence(ctx, ev, RC.GAMMA)
    for prec, tol in ((M.FP64, RC.phase_floor(ph, ev)), (M.FP32, TOL32)):
        got = M.simulate_coils(ctx, p, s, sens, prec)
        ctx.stream_status()
        assert rel_l2(got, ref) <= tol


def test_rewound_snapshots_parity(M, ctx, oracle_mod):
    ev = RC.flash_like(n_tr=20, n_read=32)
    per_tr = len(ev) // 20
    snaps = np.array([2 * per_tr + 1, 9 * per_tr + 6, 15 * per_tr + per_tr - 1, len(ev) - 1])
    assert RC.fold_counts(M, ev, snapshots=snaps)[0] == 18
    ph = RC.phantom(900 + 11, np.random.default_rng(23))
    p = M.Phantom.from_workload_phantom(ctx, ph)
    s = M.Sequence(ctx, ev, RC.GAMMA, snapshots=snaps)
    ref_sig, _ = oracle_mod.simulate(ph, ev, RC.GAMMA)
    refs = [oracle_mod.simulate(ph, ev[: e + 1], RC.GAMMA, want_signal=False, want_state=True)[1] for e in snaps]
    tol64 = RC.phase_floor(ph, ev)
    for prec in (M.FP64, M.FP32):
        out = np.zeros((len(snaps), ph.n, 3))
        sig = M.simulate(ctx, p, s, prec, snapshots=out)
        ctx.stream_status()
        tol_s, tol_m = (tol64, tol64) if prec == M.FP64 else (TOL32, 1e-4)
        assert rel_l2(sig, ref_sig) <= tol_s
        for q in range(len(snaps)):
            assert np.max(np.abs(out[q] - refs[q])) <= tol_m * (max(1.0, np.abs(refs[q]).max()) if prec == M.FP64 else 1.0), q
