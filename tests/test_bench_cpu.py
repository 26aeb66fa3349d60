"""The benchmark's host side without a GPU: the reference arm's JSON line (the oracle on the host
cores), the algorithmic work model behind the roofline, the traffic-record lookup, and that the
GPU arm refuses to run without a GPU instead of falling back to the CPU."""
import importlib.util
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def _run(args, env=None, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout, env=dict(os.environ, **(env or {})))


def test_reference_arm_line(oracle_mod):
    r = _run(["--impl", "reference", "--workload", "c1", "--steps", "1", "--warmup", "3", "--ref-seconds", "0.3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "gpu_launches"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["warmup"] >= 3 and d["steps"] == 1 and d["vs_baseline"] is None
    assert d["config"]["workload"] == "c1_flash2d_64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    r = _run(["--impl", "reference", "--workload", "c1", "--steps", "1"], env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_gpu_arm_has_no_cpu_fallback():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run(["--workload", "c1", "--steps", "1", "--warmup", "3", "--no-cpu-baseline"], timeout=300)
    assert r.returncode != 0
    assert not any(ln.startswith("{") for ln in r.stdout.splitlines())


def test_algorithmic_work_model(bench):
    rows = [(1e-5, 0, 0, 0, 0.3, 0, 0, 0.0),   # RF: 10
            (1e-5, 1e-3, 0, 0, 0, 0, 1, 0.0),  # sample: 6
            (1e-5, 1e-3, 0, 0, 0, 0, 1, 0.0),  # sample: 6
            (1e-3, 0, 0, 0, 0, 0, 0, 0.0),     # free: 4
            (1e-5, 0, 0, 0, 0.2, 0, 1, 0.0)]   # RF and sample in one event: 6 + 10 - 4 + 2
    ev = W.make_events(rows)
    assert bench.algorithmic_ops_per_spin(ev) == 10 + 6 + 6 + 4 + 14
    # with receive coils a sample costs the precession plus one weighted sum per coil
    assert bench.algorithmic_ops_per_spin(ev, n_coils=3) == 10 + 2 * 16 + 4 + (16 + 10 - 4 + 2)
    # the per-event model: RF 9; a sample that repeats the previous event's (G, dt) 7, one that does
    # not 12; any other event 12; plus 3/k per sample for k spins per thread
    assert bench.per_event_ops_per_spin(ev, 4) == 9 + 12 + 7 + 12 + 9 + 3 * 3 / 4
    assert bench.per_event_ops_per_spin(ev, 1) == 9 + 12 + 7 + 12 + 9 + 3 * 3
    # C2's mix: 65 280 repeating and 256 other samples, 65 536 sub-pulses, 1 536 other events
    w2 = W.config2()
    ev2 = w2.sequence.events
    per = bench.per_event_ops_per_spin(ev2, 8) / len(ev2)
    n_adc = int(np.count_nonzero(ev2["adc"]))
    n_rf = int(np.count_nonzero(ev2["rf_flip"] != 0))
    assert n_adc == 65536 and n_rf == 65536
    assert abs(per - (7 * (n_adc - 256) + 12 * (256 + len(ev2) - n_adc - n_rf) + 9 * n_rf + 3 / 8 * n_adc) / len(ev2)) < 1e-12
    # a rasterized list has more events but the same canonical work (the roofline uses the latter)
    w = W.config1()
    r = bench.rasterized(w, 1e-5)
    assert r.name == "c1_flash2d_64_rasterized10us" and r.sequence.n_events == 64000
    assert r.phantom is w.phantom


def test_traffic_records_follow_the_kernel_source(bench):
    rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    for name, e in rec.items():
        ps = e.get("program_sha")
        assert bench.traffic_for(e["kernel_source_sha"], name, ps) == e["dram_bytes_per_launch"]
        assert bench.traffic_for("0" * 16, name, ps) is None
        if ps is not None:  # a program-driven kernel's record also needs the program's structure
            assert bench.traffic_for(e["kernel_source_sha"], name, "0" * 16) is None
            assert bench.traffic_for(e["kernel_source_sha"], name) is None
        assert e["dram_bytes_per_launch"] == e["dram_read_bytes"] + e["dram_write_bytes"]
        assert "--clock-control none" in e["source"]
    # the hash ignores comments and whitespace only
    assert len(bench.kernel_source_sha()) == 16 and bench.kernel_source_sha() != bench.kernel_source_sha(bench.KT_SOURCES)


def test_traffic_record_matches_the_committed_compiler(bench):
    """The C2 record holds for the program the committed host compiler makes of C2, and the
    program hash sees a structural change (one sample fewer) but not a change of payload (another
    receiver phase)."""
    from paper_1305_6861_gb300 import mrsim as M

    rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))["c2_se2d_256"]
    seq = W.config2().sequence
    assert bench.program_sha(M, [seq]) == rec["program_sha"]
    assert bench.kernel_source_sha() == rec["kernel_source_sha"]
    ev = seq.events.copy()
    adc = np.nonzero(ev["adc"])[0]
    ev["adc_phase"][adc] += 0.25
    assert bench.program_sha(M, [W.Sequence(ev, seq.gamma_hz_per_t)]) == rec["program_sha"]
    ev["adc"][adc[-1]] = 0
    assert bench.program_sha(M, [W.Sequence(ev, seq.gamma_hz_per_t)]) != rec["program_sha"]


def test_field_work_model(bench):
    """Cached-map model of the non-parallel-field step: an interval computed from its record 81
    (+42 with transverse components), an interval equal to the held one 9, a pulse 9, a sample 4;
    events of zero length cost no free step; the anchored steps of a run are computed."""
    rows = [(1e-5, 0, 0, 0, 0.3, 0, 0, 0.0),    # pulse + new interval: 9 + 81
            (1e-5, 0, 0, 0, 0.3, 0, 0, 0.0),    # pulse + the same interval: 9 + 9
            (1e-5, 1e-3, 0, 0, 0, 0, 1, 0.0),   # new interval (transverse) + sample: 81 + 42 + 4
            (0.0, 0, 0, 0, 0.2, 0, 1, 0.0)]     # pulse + sample, no interval: 9 + 4
    ev = W.make_events(rows)
    gt = np.zeros((4, 6))
    gt[2, 0] = 1e-3
    assert bench.field_ops_per_spin(ev, gt) == (9 + 81) + (9 + 9) + (81 + 42 + 4) + (9 + 4)
    # without transverse components the third interval is still new (its G differs)
    assert bench.field_ops_per_spin(ev, None) == (9 + 81) + (9 + 9) + (81 + 4) + (9 + 4)
    # a readout run of 70 equal intervals: the first computed, steps 32 and 64 and the last (70)
    # anchored, the other 66 repeat the first
    ro = W.make_events([(1e-5, 1e-3, 0, 0, 0, 0, 1, 0.0)] * 70)
    computed, repeat = bench.field_event_classes(ro, None)
    assert np.flatnonzero(computed).tolist() == [0, 31, 63, 69] and np.count_nonzero(repeat) == 66
    assert bench.field_ops_per_spin(ro, None) == 4 * 81 + 66 * 9 + 70 * 4
