"""Host-side checks without a GPU: the library's exports, its input validation, and the
sequence compiler (the compiled program, interpreted on the CPU, must reproduce the oracle)."""
import math
import re
import os
import ctypes

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W
from program_interp import interpret

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def test_library_exports_every_declared_symbol(mrsim_lib):
    header = open(os.path.join(ROOT, "include", "mrsim.h")).read()
    declared = set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(mrsim_[a-z_0-9]+)\s*\(", header, re.M))
    assert declared, "no declarations parsed"
    assert declared == set(mrsim_lib.EXPORTS), f"header/binding drift: {declared ^ set(mrsim_lib.EXPORTS)}"
    L = mrsim_lib.lib()
    for name in declared:
        assert hasattr(L, name), f"{name} not exported"


def test_status_strings(mrsim_lib):
    L = mrsim_lib.lib()
    for s in range(6):
        assert L.mrsim_status_string(s)


def _compile_rc(events, gamma=W.GAMMA_BAR):
    L = __import__("paper_1305_6861_gb300.mrsim", fromlist=["x"]).lib()
    ev = np.ascontiguousarray(events, dtype=W.EVENT_DTYPE)
    from paper_1305_6861_gb300 import mrsim as M

    d = M.ProgramDump()
    return L.mrsim_debug_compile(ev.shape[0], ctypes.c_void_p(ev.ctypes.data), float(gamma), ctypes.byref(d))


@pytest.mark.parametrize("field,value", [("dt", -1e-3), ("gx", np.nan), ("rf_flip", np.inf), ("adc", 2),
                                         ("reserved", 1), ("adc_phase", np.nan)])
def test_invalid_events_rejected(mrsim_lib, field, value):
    ev = W.make_events([(1e-3, 0, 0, 0, 0.5, 0, 1, 0.0)] * 3)
    ev[field][1] = value
    assert _compile_rc(ev) == 1  # MRSIM_EINVAL


def test_invalid_gamma_rejected(mrsim_lib):
    ev = W.make_events([(1e-3, 0, 0, 0, 0.5, 0, 1, 0.0)])
    assert _compile_rc(ev, 0.0) == 1
    assert _compile_rc(ev, -1.0) == 1
    assert _compile_rc(ev, np.nan) == 1
    assert _compile_rc(ev[:0]) == 0


def test_context_without_gpu_is_unsupported(mrsim_lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert mrsim_lib.lib().mrsim_context_create(0, ctypes.byref(h)) == 5  # MRSIM_EUNSUPPORTED


def _check_structure(events, ops, n_adc):
    from paper_1305_6861_gb300 import mrsim as M

    assert len(ops) <= 2 * len(events) + 1  # an event with RF and a sample is two ops
    assert ops[-1]["kind"] == M.OP_END
    seen = []
    for op in ops:
        if op["kind"] == M.OP_RF_TRAIN:
            continue
        if op["kind"] == M.OP_RUN:
            assert 1 <= op["n"] <= 256
            seen.extend(range(op["adc0"], op["adc0"] + op["n"]))
        elif op["flags"] & M.F_ADC:
            seen.append(op["adc0"])
    assert seen == list(range(n_adc)), "every sample exactly once, in order"


CASES = {
    "c1": lambda: W.config1(),
    "c2_small": lambda: W.config2(n=32, iso=2),
    "c3_small": lambda: W.config3(n=12, iso=1),
    "c5_small": lambda: W.config5(n=24)[0],
}


@pytest.mark.parametrize("case", list(CASES))
def test_compiled_program_matches_oracle(case, mrsim_lib, oracle_mod):
    w = CASES[case]()
    seq = w.sequence
    sig, state, ops = interpret(seq.events, seq.gamma_hz_per_t, w.phantom)
    ref, ref_state = oracle_mod.simulate(w.phantom, seq.events, seq.gamma_hz_per_t, want_state=True)
    _check_structure(seq.events, ops, seq.n_adc)
    assert rel_l2(sig, ref) < 1e-12
    assert np.max(np.abs(state - ref_state)) < 1e-12 * max(1.0, np.max(np.abs(ref_state)))


@pytest.mark.parametrize("seed", range(6))
def test_compiled_random_programs_match_oracle(seed, mrsim_lib, oracle_mod):
    rng = np.random.default_rng(100 + seed)
    ph = W.random_phantom(50, rng)
    seq = W.random_sequence(400, rng, runs=seed % 3 != 0)
    m0 = rng.normal(size=(ph.n, 3)) if seed % 2 else None
    sig, state, ops = interpret(seq.events, seq.gamma_hz_per_t, ph, state_in=m0)
    ref, ref_state = oracle_mod.simulate(ph, seq.events, seq.gamma_hz_per_t, m_init=m0, want_state=True)
    _check_structure(seq.events, ops, seq.n_adc)
    assert rel_l2(sig, ref) < 1e-11
    assert np.max(np.abs(state - ref_state)) < 1e-11 * max(1.0, np.max(np.abs(ref_state)))


def test_class_tables_bounded_and_used(mrsim_lib):
    from paper_1305_6861_gb300 import mrsim as M

    w = W.config2(n=32, iso=2)
    prog = M.debug_compile(w.sequence.events, w.sequence.gamma_hz_per_t)
    ops = prog["ops"]
    assert len(prog["pcls"]) <= 8 and len(prog["e1"]) <= 4 and len(prog["e2"]) <= 4
    # every shaped pulse is a few general RF operations (frame turn, cache loads, the unfused last
    # excitation sub-pulse) plus one train operation over the sub-pulse table; the two distinct
    # pulse shapes (90° and 180°) are stored once and shared by all TRs
    trains = ops[ops["kind"] == M.OP_RF_TRAIN]
    assert len(trains) == 2 * 32
    assert np.count_nonzero(ops["kind"] == M.OP_RF) <= 6 * 32
    assert len(prog["train"]) == sum(sorted(set(zip(trains["adc0"], trains["n"])), key=lambda t: t[0])[i][1] for i in range(2))
    assert len(prog["train"]) < 2 * 128
    # every readout is one run with an anchor
    runs = ops[ops["kind"] == M.OP_RUN]
    assert len(runs) == 32 and np.all(runs["flags"] & M.F_ANCHOR)


@pytest.mark.parametrize("seed", range(3))
def test_snapshots_compiled_program(oracle_mod, mrsim_lib, seed):
    """Snapshots (§7.2) after chosen events: the compiled program's states equal the oracle's final
    state on the event prefix, and the signal is unchanged by them."""
    rng = np.random.default_rng(4200 + seed)
    ph = W.random_phantom(300, rng)
    seq = W.random_sequence(700, rng, runs=True)
    ev = seq.events
    snaps = np.sort(rng.choice(len(ev), size=6, replace=False))
    snaps[-1] = len(ev) - 1
    M = mrsim_lib
    sig, state, ops, got = interpret(ev, seq.gamma_hz_per_t, ph, snapshots=snaps)
    assert np.count_nonzero(ops["kind"] == M.OP_SNAP) == len(snaps)
    # float64 floor for phases of ~1e4 rad per event: each side rounds θ with relative error 2^-53
    g = 2 * math.pi * seq.gamma_hz_per_t
    th = (g * (np.abs(ev["gx"]) * np.abs(ph.x).max() + np.abs(ev["gy"]) * np.abs(ph.y).max()
               + np.abs(ev["gz"]) * np.abs(ph.z).max()) + np.abs(ph.dw).max()) * ev["dt"]
    tol = max(1e-12, 4 * 2.0**-53 * float(np.sqrt(np.sum(th**2))))
    ref_sig, _ = oracle_mod.simulate(ph, ev, seq.gamma_hz_per_t)
    assert np.linalg.norm(sig - ref_sig) <= tol * np.linalg.norm(ref_sig)
    for q, e in enumerate(snaps):
        _, st = oracle_mod.simulate(ph, ev[: e + 1], seq.gamma_hz_per_t, want_signal=False, want_state=True)
        assert np.max(np.abs(got[q] - st)) <= tol * max(1.0, np.abs(st).max()), (q, e)
    assert np.max(np.abs(got[-1] - state)) <= 1e-13


def test_snapshot_lists_are_validated(mrsim_lib):
    ev = W.random_sequence(50, np.random.default_rng(3)).events
    for bad in ([5, 5], [7, 3], [-1], [50]):
        with pytest.raises(mrsim_lib.MrsimError) as e:
            mrsim_lib.debug_compile(ev, W.GAMMA_BAR, snapshots=bad)
        assert e.value.status == mrsim_lib.Status.EINVAL


# ---- rewound readouts: A (phase encoding), run, B (rewinder) folded into the run ----------------
import rewound_cases as RC


def _fold_check(M, oracle_mod, ev, ph, snapshots=None):
    out = interpret(ev, RC.GAMMA, ph, snapshots=snapshots)
    sig, state, ops = out[:3]
    ref, ref_state = oracle_mod.simulate(ph, ev, RC.GAMMA, want_state=True)
    _check_structure(ev, ops, int(np.count_nonzero(ev["adc"])))
    tol = RC.phase_floor(ph, ev)
    assert rel_l2(sig, ref) <= tol
    assert np.max(np.abs(state - ref_state)) <= tol * max(1.0, np.max(np.abs(ref_state)))
    return out


@pytest.mark.parametrize("case", ["c1", "c3_small"])
def test_gradient_echo_readouts_are_folded(case, mrsim_lib):
    """Every readout of the gradient-echo configurations folds its phase encoding and rewinder:
    no inline precession op is left and each TR is one pulse and one run."""
    M = mrsim_lib
    w = CASES[case]()
    ops = M.debug_compile(w.sequence.events, w.sequence.gamma_hz_per_t)["ops"]
    runs = ops[ops["kind"] == M.OP_RUN]
    assert len(runs) > 0 and np.all(runs["flags"] & M.F_INLINE) and np.all(runs["flags"] & M.F_ANCHOR)
    assert not np.any((ops["kind"] == M.OP_PREC) & ((ops["flags"] & M.F_INLINE) != 0))


def test_fold_program_matches_oracle(mrsim_lib, oracle_mod):
    ev = RC.flash_like()
    assert RC.fold_counts(mrsim_lib, ev) == (16, 16, 0)
    _fold_check(mrsim_lib, oracle_mod, ev, RC.phantom(80, np.random.default_rng(7)))


def test_no_fold_when_the_rewinder_misses(mrsim_lib, oracle_mod):
    """A rewinder that leaves a different residual moment every TR gives no recurring total, so
    nothing is folded (the readout keeps its own anchor) and the program is unchanged in meaning."""
    ev = RC.flash_like(jitter=np.random.default_rng(3))
    folded, runs, inline = RC.fold_counts(mrsim_lib, ev)
    assert folded == 0 and runs == 16 and inline == 32
    _fold_check(mrsim_lib, oracle_mod, ev, RC.phantom(60, np.random.default_rng(8)))


def test_no_rewinder_no_fold(mrsim_lib, oracle_mod):
    ev = RC.flash_like(rewind=False)
    assert RC.fold_counts(mrsim_lib, ev)[0] == 0
    _fold_check(mrsim_lib, oracle_mod, ev, RC.phantom(60, np.random.default_rng(9)))


def test_overlapping_triples_fold_once(mrsim_lib, oracle_mod):
    """Multi-echo readouts: A+R1+B and B+R2+C both recur; B can only belong to one fold, so the
    first readout of each TR folds and the second keeps its plain anchor."""
    ev = RC.multi_echo()
    folded, runs, inline = RC.fold_counts(mrsim_lib, ev)
    assert (folded, runs, inline) == (12, 24, 12)
    _fold_check(mrsim_lib, oracle_mod, ev, RC.phantom(70, np.random.default_rng(10)))


def test_snapshot_inside_a_rewound_readout(mrsim_lib, oracle_mod):
    """A snapshot between the phase encoding and the readout (or inside the readout) needs the
    state there: that TR is not folded, the others are."""
    M = mrsim_lib
    ev = RC.flash_like()
    per_tr = len(ev) // 16
    snaps = np.array([3 * per_tr + 1, 7 * per_tr + 5, len(ev) - 1])  # after A of TR 3; inside R of TR 7
    folded, runs, _ = RC.fold_counts(M, ev, snapshots=snaps)
    assert runs >= 16 and folded == 14
    ph = RC.phantom(50, np.random.default_rng(11))
    _, _, _, got = _fold_check(M, oracle_mod, ev, ph, snapshots=snaps)
    tol = RC.phase_floor(ph, ev)
    for q, e in enumerate(snaps):
        _, st = oracle_mod.simulate(ph, ev[: e + 1], RC.GAMMA, want_signal=False, want_state=True)
        assert np.max(np.abs(got[q] - st)) <= tol * max(1.0, np.abs(st).max()), q


# ---- context-free compilation (mrsim_compile) -------------------------------------------------
def test_compile_without_context(mrsim_lib):
    """mrsim_compile needs no GPU; its upload size is the program the debug dump describes."""
    M = mrsim_lib
    w = CASES["c2_small"]()
    c = M.Compiled(w.sequence.events, w.sequence.gamma_hz_per_t)
    d = M.debug_compile(w.sequence.events, w.sequence.gamma_hz_per_t)
    n_adc, n_tr = len(d["demod"]), len(d["train"])
    assert c.n_adc == n_adc == w.sequence.n_adc
    n_tmap = len({int(o["tab"]) for o in d["ops"] if o["kind"] == M.OP_RF_TRAIN and o["flags"] & M.F_TMAP})
    tables = [len(d["ops"]) * 64, len(d["ops"]) * 128, 8 * d["pcls"].size, 8 * d["e1"].size, 8 * d["e2"].size,
              16 * n_adc, 8 * n_adc, 8 * n_tr, 16 * n_tr, 16 * n_tmap]  # one image, tables on 256-byte boundaries
    assert c.upload_bytes == sum(-(-b // 256) * 256 for b in tables)
    c.close()
    c.close()  # idempotent


def test_compile_errors_are_per_thread(mrsim_lib):
    import threading

    M = mrsim_lib
    good = W.config1().sequence.events
    bad = W.make_events([(1e-3, 0, 0, 0, 0.5, 0, 1, 0.0)] * 3)
    bad["dt"][1] = -1.0
    msgs = {}

    def run(name, ev):
        try:
            M.Compiled(ev, W.GAMMA_BAR).close()
            msgs[name] = M.lib().mrsim_compile_last_error().decode()
        except M.MrsimError as e:
            msgs[name] = str(e)

    ts = [threading.Thread(target=run, args=("bad", bad)), threading.Thread(target=run, args=("good", good))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert "negative duration" in msgs["bad"] and msgs["good"] == ""


def test_concurrent_compiles_are_identical(mrsim_lib):
    """Compilation keeps no shared state: programs compiled on several threads at once match the
    serial one field by field."""
    from concurrent.futures import ThreadPoolExecutor

    M = mrsim_lib
    seqs = [CASES["c2_small"]().sequence.events, W.config1().sequence.events,
            W.random_sequence(3000, np.random.default_rng(77)).events, RC.flash_like()]
    gammas = [W.GAMMA_BAR, W.GAMMA_BAR, W.GAMMA_BAR, RC.GAMMA]
    ref = [M.debug_compile(e, g) for e, g in zip(seqs, gammas)]
    with ThreadPoolExecutor(8) as pool:
        got = list(pool.map(lambda i: M.debug_compile(seqs[i % 4], gammas[i % 4]), range(32)))
    for i, d in enumerate(got):
        r = ref[i % 4]
        for k in r:
            assert np.array_equal(r[k].view(np.uint8), d[k].view(np.uint8)), (i, k)


def test_compile_argument_checks(mrsim_lib):
    import ctypes

    L = mrsim_lib.lib()
    ev = np.ascontiguousarray(W.config1().sequence.events)
    assert L.mrsim_compile(ev.shape[0], ctypes.c_void_p(ev.ctypes.data), W.GAMMA_BAR, 0, None, None) == 1
    assert "NULL" in L.mrsim_compile_last_error().decode()
    h = ctypes.c_void_p()
    assert L.mrsim_compile(ev.shape[0], ctypes.c_void_p(ev.ctypes.data), W.GAMMA_BAR, 0, None, ctypes.byref(h)) == 0
    assert L.mrsim_compile_last_error().decode() == "" and L.mrsim_compiled_num_adc(h) == 4096
    L.mrsim_compiled_destroy(h)
    assert L.mrsim_compiled_num_adc(None) == -1 and L.mrsim_compiled_upload_bytes(None) == -1
    L.mrsim_compiled_destroy(None)
    snaps = np.array([5, 3], dtype=np.int64)  # not increasing
    assert L.mrsim_compile(ev.shape[0], ctypes.c_void_p(ev.ctypes.data), W.GAMMA_BAR, 2,
                           ctypes.c_void_p(snaps.ctypes.data), ctypes.byref(h)) == 1


def test_log_callback_and_env(mrsim_lib):
    """Failed calls reach the log callback (here: mrsim_compile, which needs no GPU) and, with
    MRSIM_LOG set, stderr."""
    import ctypes
    import subprocess
    import sys

    L = mrsim_lib.lib()
    got = []
    FN = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.c_char_p, ctypes.c_void_p)
    cb = FN(lambda st, msg, user: got.append((st, msg.decode())))
    L.mrsim_set_log_callback(ctypes.cast(cb, ctypes.c_void_p), None)
    try:
        bad = W.make_events([(1e-3, 0, 0, 0, 0.5, 0, 1, 0.0)] * 2)
        bad["dt"][0] = -1.0
        with pytest.raises(mrsim_lib.MrsimError):
            mrsim_lib.Compiled(bad, W.GAMMA_BAR)
    finally:
        L.mrsim_set_log_callback(None, None)
    assert got and got[-1][0] == 1 and "negative duration" in got[-1][1]
    code = ("import numpy as np\n"
            "from paper_1305_6861_gb300 import mrsim as M, workloads as W\n"
            "ev = W.make_events([(1e-3, 0, 0, 0, 0.5, 0, 1, 0.0)]); ev['adc'][0] = 3\n"
            "try:\n    M.Compiled(ev, W.GAMMA_BAR)\nexcept M.MrsimError:\n    pass\n")
    env = dict(os.environ, MRSIM_LOG="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "mrsim: invalid argument: event 0: adc must be 0/1" in r.stderr


def test_train_map_kinds(mrsim_lib):
    """The compiler marks a shaped pulse that recurs (at least 4 times with the same sub-pulse
    flips, precession class and T1 class) as a train-map kind: C2's two sinc pulses, 256
    occurrences each, 125 fast sub-pulses each; C1 (hard pulses) has none; a train that occurs
    once is not mapped."""
    M = mrsim_lib

    def kinds(events, gamma):
        ops = M.debug_compile(events, gamma)["ops"]
        out = {}
        for o in ops[(ops["kind"] == M.OP_RF_TRAIN) & ((ops["flags"] & M.F_TMAP) != 0)]:
            out.setdefault(int(o["tab"]), [int(o["n"]), 0])[1] += 1
        return out

    w2 = W.config2()
    assert sorted(kinds(w2.sequence.events, w2.sequence.gamma_hz_per_t).values()) == [[125, 256], [125, 256]]
    w1 = W.config1()
    assert kinds(w1.sequence.events, w1.sequence.gamma_hz_per_t) == {}
    one = W.spin_echo(16, 8, 0.5, 12e-3, 30e-3, 10e-6, n_rf=24)
    ev = one.events[: len(one.events) // 16]  # a single TR: every train occurs once
    assert kinds(ev, one.gamma_hz_per_t) == {}
    assert len(kinds(one.events, one.gamma_hz_per_t)) >= 1

