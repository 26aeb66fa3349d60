"""Benchmark: spin-steps/s of the forward simulation on GB300 (one JSON line on rank 0).

A step is one forward simulation (all operations of the hot path: RF rotations, precession and
relaxation of every spin through every event, and the per-sample signal sum) of the workload's
phantom through its sequence, with inputs resident in device memory.  Default workload: the
3D 128³ RF-spoiled gradient echo (2 isochromats/voxel, 4 194 304 spins, 2 146 304 events;
`--workload c3`); `--workload c1|c2|c4|c5|kt` gives the others.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3|c2|c1|c4|c5|kt] [--impl ours|reference]

N > 1 (torchrun): weak scaling — every rank simulates its own phantom of the workload's size
(a different seed), the ranks' phantoms form one object, and the per-step exchange is the
sum-reduce of the complex signal over ranks (NCCL all-reduce).

Roofline: FP32 lane-operations of the per-event model (an ADC event that repeats the previous
event's gradient and duration 7, an RF event 9, any other event 12, plus 3/k per sample for the
shared-memory transpose of k spins per thread) per launch, over the kernel's CUDA-event time,
against SMs (read from the device) x 128 FP32 lanes x the SM clock sampled during the timed
region.  Beside it: the stricter formulation model (the arithmetic the pulse-frame formulation
needs) and the multiply-add rates a probe kernel measures on the same device in the same run
(float32, float32 pairs, float64; the float64 figure is the float64 path's peak).

Oracle parity: the float64 CPU oracle on a seeded spin sample (1 % of C3's spins by default)
against the GPU signal of the same spins taken from a launch of the whole phantom in the timed
launch shape, with every other spin's M0 set to zero (their contribution is exactly zero), so
the sample runs through the benchmark's own blocks and cross-block sums.

The reference arm (`--impl reference`) times the FP64 CPU oracle on the host cores, on a
bounded spin sample of the same workload.

`--raster 1e-5` is a stress mode for c1-c3: every event is cut into pieces of at most 10 µs (the
"piecewise-constant 10 µs events" reading of the event lists), the signal is the same, and the
spin-step count is that of the pieces; the line is labelled `stress_mode` in its config.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1305_6861_gb300 import workloads as W  # noqa: E402
from paper_1305_6861_gb300 import distributed as D  # noqa: E402

METRIC = "spin-steps/s (isochromat×event updates) at 1 GB300, FP32 vs FP64, % FP32/SFU peak"
# FP32 lane-operations the method needs per spin-step, by event type (pulse-frame formulation):
#   ADC event: precession-relaxation of Mxy, one complex product (4) + accumulate into the sample (2)
#   RF event : hard pulse in its own frame (4) + T1 recovery of Mz (2) + precession (4)
#   other    : precession (4); T1 recovery is folded into the next pulse
OPS_ADC, OPS_RF, OPS_OTHER = 6, 10, 4
# Per-event model of the FP32 work per spin-step (FMA = 1): an ADC event that repeats the previous
# event's (G, Δt) reuses the spin's rotation factor (7), an RF event is the 3x3 rotation (9), any
# other event is a precession-relaxation with a fresh phase (12); each sample also costs 3/k for
# the shared-memory transpose of its partial sums with k spins per thread.
EV_ADC_REPEAT, EV_RF, EV_OTHER, EV_SAMPLE_TRANSPOSE = 7, 9, 12, 3
# A recurring shaped pulse run as its train map: per occurrence the 3x3 map and offset (12) in place
# of its sub-pulses; per kind, once per launch, four states stepped through its sub-pulses.
EV_MAP = 12
FP32_LANES = 128      # FP32 lanes per SM (unit count)
SM_MAX_MHZ = 2070.0   # used only when no clock sample exists


def algorithmic_ops_per_spin(events, n_coils: int = 0) -> int:
    """FP32 lane-ops per spin over the sequence; with receive coils a sample costs the precession
    (4) plus one weighted complex accumulation per coil (4, the sum folded into the FMAs)."""
    ops_adc = OPS_ADC if n_coils == 0 else 4 + 4 * n_coils
    adc = events["adc"] != 0
    rf = (events["rf_flip"] != 0) & ~adc
    other = ~adc & ~rf
    n_rf_adc = int(np.count_nonzero((events["rf_flip"] != 0) & adc))
    return int(ops_adc * np.count_nonzero(adc) + OPS_RF * np.count_nonzero(rf) + OPS_OTHER * np.count_nonzero(other)
               + (OPS_RF - OPS_OTHER + 2) * n_rf_adc)


def ring_coils(phantom, n_coils: int, radius: float = 0.3, width: float = 0.25):
    """Synthetic array-coil sensitivities: Gaussian magnitude around n coils on a ring, phase
    growing along the ring; complex [n_coils, n_spins]."""
    ang = 2 * math.pi * np.arange(n_coils) / n_coils
    cx, cy = radius * np.cos(ang), radius * np.sin(ang)
    d2 = (phantom.x[None, :] - cx[:, None]) ** 2 + (phantom.y[None, :] - cy[:, None]) ** 2
    return np.exp(-d2 / width**2) * np.exp(1j * (ang[:, None] + 4.0 * phantom.x[None, :] * np.cos(ang)[:, None]))


def per_event_ops_per_spin(events, spins_per_thread: int) -> float:
    """FP32 lane-ops per spin over the sequence by the per-event model (EV_*)."""
    ev = events
    adc = ev["adc"] != 0
    rf = ev["rf_flip"] != 0
    same = np.zeros(len(ev), dtype=bool)
    if len(ev) > 1:
        same[1:] = ((ev["dt"][1:] == ev["dt"][:-1]) & (ev["gx"][1:] == ev["gx"][:-1])
                    & (ev["gy"][1:] == ev["gy"][:-1]) & (ev["gz"][1:] == ev["gz"][:-1]))
    n_rf = int(np.count_nonzero(rf))
    n_adc_rep = int(np.count_nonzero(adc & ~rf & same))
    n_other = len(ev) - n_rf - n_adc_rep
    return (EV_RF * n_rf + EV_ADC_REPEAT * n_adc_rep + EV_OTHER * n_other
            + EV_SAMPLE_TRANSPOSE / max(int(spins_per_thread), 1) * int(np.count_nonzero(adc)))


def train_map_kinds(M, events, gamma_hz_per_t) -> list:
    """The compiled program's train maps: per kind, (sub-pulses, occurrences)."""
    ops = M.debug_compile(events, gamma_hz_per_t)["ops"]
    kinds = {}
    for o in ops[(ops["kind"] == M.OP_RF_TRAIN) & ((ops["flags"] & M.F_TMAP) != 0)]:
        kinds.setdefault(int(o["tab"]), [int(o["n"]), 0])[1] += 1
    return [tuple(v) for v in kinds.values()]


def map_adjusted(ops_per_spin: float, per_sub: float, kinds) -> float:
    """A model's ops per spin when the recurring trains run as maps: each occurrence applies its
    map (EV_MAP) instead of its n sub-pulses (per_sub each), and each kind's map is formed once by
    stepping four states (the three unit states and the zero state) through its n sub-pulses."""
    return ops_per_spin + sum(occ * (EV_MAP - per_sub * n) + 4 * per_sub * n for n, occ in kinds)


# Device facts and measured rates, filled by measure_device() before any timed region.
DEVICE = {"sms": None, "fp32_lane_ops_per_s": None, "fp32x2_lane_ops_per_s": None, "fp64_lane_ops_per_s": None,
          "probe_sm_mhz": None}


def measure_device(ctx, M, device: int, stream=None) -> dict:
    """SM count from the device, and the multiply-add rates the library's probe kernel reaches on
    it (float32, float32 pairs, float64; about 0.3 s each), with the SM clock sampled meanwhile."""
    import torch

    DEVICE["sms"] = torch.cuda.get_device_properties(device).multi_processor_count
    ck = ClockSampler(device, tag="probe")
    ck.start()
    time.sleep(0.1)
    for key, kind in (("fp32_lane_ops_per_s", M.FMA_F32), ("fp32x2_lane_ops_per_s", M.FMA_F32X2),
                      ("fp64_lane_ops_per_s", M.FMA_F64)):
        DEVICE[key] = M.measure_fma_rate(ctx, kind, 300.0, stream=stream)[0]
    DEVICE["probe_sm_mhz"] = ck.stop().get("sm_mhz")
    return dict(DEVICE)


def sm_clock(ck: dict) -> float:
    """The SM clock of a peak: the median sampled under load in the timed region, else the maximum."""
    return float(ck.get("sm_mhz") or ck.get("sm_max_mhz") or SM_MAX_MHZ)


def fp32_alu_peak_ops(sm_mhz: float) -> float:
    """Unit-count FP32 rate: SMs (from the device) x 128 lanes x the SM clock."""
    return DEVICE["sms"] * FP32_LANES * sm_mhz * 1e6


def fp32_roofline(achieved_g: float, ck: dict, **extra) -> dict:
    """FP32 lane-ops against the unit-count peak at the sampled clock, and against the measured
    float32 multiply-add rate of the same device."""
    mhz = sm_clock(ck)
    peak = fp32_alu_peak_ops(mhz) / 1e9
    r = {"bound": "alu", "achieved": achieved_g, "peak": peak, "unit": "G FP32 lane-ops/s", "frac": achieved_g / peak,
         "peak_basis": f"{DEVICE['sms']} SMs (device) x {FP32_LANES} FP32 lanes x {mhz:.0f} MHz (median SM clock "
                       "sampled in the timed region)"}
    r.update(extra)
    meas = max(DEVICE["fp32_lane_ops_per_s"] or 0.0, DEVICE["fp32x2_lane_ops_per_s"] or 0.0) / 1e9
    if meas:
        r["measured_fma"] = {"peak": meas, "frac": achieved_g / meas, "sm_mhz": DEVICE["probe_sm_mhz"],
                             "basis": "float32 multiply-add chains (scalar or pairs, the faster) on every SM, "
                                      "CUDA-event timed in this run"}
    return r


def fp64_roofline(achieved_g: float) -> dict:
    """Algorithmic lane-ops of a float64 run against the float64 multiply-add rate measured on the
    same device in the same run (G lane-ops/s)."""
    peak = DEVICE["fp64_lane_ops_per_s"] / 1e9
    return {"bound": "fp64", "achieved": achieved_g, "peak": peak, "unit": "G float64 lane-ops/s",
            "frac": achieved_g / peak, "traffic": None,
            "peak_basis": "float64 multiply-add chains on every SM, CUDA-event timed in this run "
                          f"(SM clock {DEVICE['probe_sm_mhz']} MHz)"}


def measured_rates() -> dict:
    return {"sms": DEVICE["sms"], "sm_mhz": DEVICE["probe_sm_mhz"],
            "fp32_G_lane_ops_per_s": (DEVICE["fp32_lane_ops_per_s"] or 0) / 1e9,
            "fp32x2_G_lane_ops_per_s": (DEVICE["fp32x2_lane_ops_per_s"] or 0) / 1e9,
            "fp64_G_lane_ops_per_s": (DEVICE["fp64_lane_ops_per_s"] or 0) / 1e9}


def build_workload(name: str, rank: int = 0):
    seed = D.rank_seed(W.SEED_BASE, {"c1": 1, "c2": 2, "c3": 3}[name], rank)
    if name == "c1":
        return W.config1(seed)
    if name == "c2":
        return W.config2(seed)
    if name == "c3":
        return W.config3(seed)
    raise ValueError(name)


def source_id() -> dict:
    """Which code produced the line: the kernel-source hash and, where the tree is a git checkout,
    the commit."""
    try:
        rev = subprocess.run(["git", "-C", ROOT, "rev-parse", "--short=12", "HEAD"], capture_output=True, text=True,
                             timeout=10).stdout.strip() or None
    except Exception:
        rev = None
    return {"fwd_kernel_source_sha": kernel_source_sha(), "kt_kernel_source_sha": kernel_source_sha(KT_SOURCES), "git": rev}


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, tag: str = "timed"):
        self.device = device
        self.proc = None
        # the raw samples go to $MRSIM_CLOCKS_DIR when set (kept beside the run's other logs)
        d = os.environ.get("MRSIM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_{tag}_rank{device}_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9 and p[1].replace(".", "").isdigit():
                rows.append(p)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [s for s in sm if s >= 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()) if rows else None}


def traffic_for(kernel_src_sha: str, workload: str, prog_sha: str | None = None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this kernel source
    and (for the program-driven kernels) on a program of this structure."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
        e = d.get(workload)
        if e and e.get("kernel_source_sha") == kernel_src_sha and e.get("program_sha") == prog_sha:
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def program_sha(M, sequences) -> str:
    """Hash of the compiled programs' structure: operation kinds, flags, counts, class and table
    indices, and the table sizes.  With the kernel source this fixes what a launch reads and
    writes; the float payloads (moments, angles, phases) are left out."""
    h = hashlib.sha256()
    for seq in sequences:
        p = M.debug_compile(seq.events, seq.gamma_hz_per_t)
        ops = p["ops"]
        for f in ("kind", "flags", "n", "adc0", "pcls", "ecls", "acls", "tab"):
            h.update(np.ascontiguousarray(ops[f]).tobytes())
        sizes = [len(ops)] + [len(p[t]) for t in ("pcls", "e1", "e2", "train", "demod")]
        h.update(np.asarray(sizes, dtype=np.int64).tobytes())
    return h.hexdigest()[:16]


# the device code of the forward and batch kernels (the program they run is hashed on its own)
FWD_SOURCES = ("fwd_kernel.cuh", "packed.cuh", "internal.h")
KT_SOURCES = ("kt_kernel.cu", "packed.cuh", "internal.h")


def kernel_source_sha(files=FWD_SOURCES) -> str:
    """Hash of the kernel sources' code (comments and whitespace removed), so that a counter
    capture stays valid across documentation edits and is dropped when the code changes."""
    import re

    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1305_6861_gb300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def cpu_baseline(w, seconds: float = 10.0, seed: int = 1):
    """The oracle, as it stands, on a bounded random spin sample of the workload (full sequence)."""
    import oracle

    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(seed)
    n_cal = min(w.phantom.n, 64)
    cal = w.phantom.subset(np.sort(rng.choice(w.phantom.n, n_cal, replace=False)))
    t0 = time.perf_counter()
    oracle.signal(cal, w.sequence, n_threads=cores)
    dt = time.perf_counter() - t0
    per_spin = dt / n_cal
    n = int(max(cores, min(w.phantom.n, seconds / max(per_spin, 1e-9))))
    sub = w.phantom.subset(np.sort(rng.choice(w.phantom.n, n, replace=False)))
    t0 = time.perf_counter()
    ref = oracle.signal(sub, w.sequence, n_threads=cores)
    el = time.perf_counter() - t0
    return {"value": n * w.sequence.n_events / el, "unit": "spin-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{w.name}: full sequence ({w.sequence.n_events} events) on {n} of {w.phantom.n} spins, {el:.1f} s"}, \
        (sub, ref)


def oracle_parity(ctx, M, w, sub, ref, n_coils: int = 0):
    """The GPU signal of the CPU baseline's spin sample in both precisions against the float64
    oracle's signal of the same spins: relative L2 and dB (the error report per configuration)."""
    p = M.Phantom.from_workload_phantom(ctx, sub)
    s = M.Sequence.from_workload_sequence(ctx, w.sequence)
    out = {"sample_spins": int(sub.n)}
    nr = float(np.linalg.norm(ref))
    for name, prec in (("fp32", M.FP32), ("fp64", M.FP64)):
        got = M.simulate(ctx, p, s, prec)
        rel = float(np.linalg.norm(got - ref) / nr) if nr > 0 else 0.0
        out[f"{name}_rel_l2"] = rel
        out[f"{name}_db"] = 20 * math.log10(rel) if rel > 0 else None
    p.close()
    s.close()
    return out


def sample_index(ph, fraction: float, seed: int = 7) -> np.ndarray:
    """Seeded sample of `fraction` of the phantom's spin count (all spins for fraction >= 1), drawn
    from the spins with M0 > 0 (air spins contribute nothing to the signal), sorted."""
    n = ph.n
    if fraction >= 1.0:
        return np.arange(n)
    m = max(1, int(round(fraction * n)))
    pool = np.nonzero(ph.rho > 0)[0]
    if pool.size < m:
        pool = np.arange(n)
    return np.sort(np.random.default_rng(seed).choice(pool, min(m, pool.size), replace=False))


def masked_phantom(ph, idx):
    """The phantom with M0 = 0 for every spin outside idx: such a spin stays at (0, 0, 0) through
    every event, so the signal is that of the sample alone while the launch covers every spin."""
    rho = np.zeros_like(ph.rho)
    rho[idx] = ph.rho[idx]
    return W.Phantom(ph.x, ph.y, ph.z, rho, ph.t1, ph.t2, ph.dw)


class OracleRun:
    """A host thread running `signal_fn(sub, sequence, n_threads=cores)` on a spin sample of a
    workload (the C oracle releases the interpreter while it runs on all host cores)."""

    def __init__(self, w, idx, signal_fn):
        import threading

        self.w, self.idx, self.fn, self.ref, self.err, self.seconds = w, idx, signal_fn, None, None, None
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def _run(self):
        try:
            sub = self.w.phantom.subset(self.idx)
            t0 = time.perf_counter()
            self.ref = self.fn(sub, self.w.sequence, n_threads=len(os.sched_getaffinity(0)))
            self.seconds = time.perf_counter() - t0
        except Exception as e:  # reported in the line
            self.err = repr(e)

    def join(self):
        self.thread.join()
        return self.ref


def cpu_baseline_parity_run(w, idx) -> OracleRun:
    """CPU-baseline leg: the float64 oracle, as it stands, on the parity sample, started on a host
    thread while the GPU legs run."""
    import oracle

    return OracleRun(w, idx, oracle.signal)


def oracle_parity_sample(ctx, M, w, run: OracleRun, seq, shape, stream=None):
    """The oracle's signal of a spin sample against the GPU's: float32 from a launch of the whole
    phantom with M0 = 0 outside the sample, in the timed launch shape (the sample's spins sit in
    the benchmark's own blocks and go through its cross-block sums); float64 from the sample
    alone."""
    ref = run.join()
    if ref is None:
        return {"error": run.err}
    out = {"sample_spins": int(run.idx.size), "of_spins": int(w.phantom.n),
           "sample_fraction": run.idx.size / max(w.phantom.n, 1), "oracle_s": run.seconds,
           "fp32_launch": f"whole phantom, M0 = 0 outside the sample, {shape[0]} spins/thread x {shape[1]} threads"}
    nr = float(np.linalg.norm(ref))
    pm = M.Phantom.from_workload_phantom(ctx, masked_phantom(w.phantom, run.idx), stream=stream)
    got32 = M.simulate(ctx, pm, seq, M.FP32, spins_per_thread=shape[0], threads_per_block=shape[1])
    pm.close()
    ps = M.Phantom.from_workload_phantom(ctx, w.phantom.subset(run.idx), stream=stream)
    got64 = M.simulate(ctx, ps, seq, M.FP64)
    ps.close()
    for name, got in (("fp32", got32), ("fp64", got64)):
        rel = float(np.linalg.norm(got - ref) / nr) if nr > 0 else 0.0
        out[f"{name}_rel_l2"] = rel
        out[f"{name}_db"] = 20 * math.log10(rel) if rel > 0 else None
    return out


def rasterized(w, raster: float):
    """The stress variant of a workload: every event cut into pieces of at most `raster` seconds
    (same signal, many more events; the spin-step count is that of the pieces)."""
    return W.Workload(w.name + f"_rasterized{raster * 1e6:g}us", w.phantom, W.rasterize(w.sequence, raster), w.note)


RASTER_NOTE = ("stress mode: every event cut into pieces of at most {r:g} us, counted as events; the host "
               "compiler merges the pieces back into the canonical program, so the roofline counts the "
               "canonical list's work ({n} events)")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = build_workload(args.workload)
    if args.raster:
        w = rasterized(w, args.raster)
    times = []
    cb = None
    for i in range(args.warmup + args.steps):
        r, _ = cpu_baseline(w, seconds=args.ref_seconds, seed=100 + i)
        if i >= args.warmup:
            times.append(r)
            cb = r
    v = statistics.median(t["value"] for t in times)
    ms = w.spin_steps / v * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "spin-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_spins": w.phantom.n, "n_events": w.sequence.n_events,
                   "note": "each step is the oracle on a bounded spin sample of the workload; ms_per_step extrapolates to the full phantom"},
        "cpu_baseline": {"value": v, "unit": "spin-steps/s", "cores": cb["cores"], "kind": "oracle", "sample": cb["sample"]},
        "e2e": {"value": v, "unit": "spin-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """Batched workload (C4): 64 phantoms / sequences in one persistent launch replayed as a CUDA
    graph.  One step = the whole batch."""
    import torch

    from paper_1305_6861_gb300 import mrsim as M

    torch.cuda.set_device(0)
    ws = W.config4()
    prec = {"fp64": M.FP64, "kahan": M.FP32_KAHAN}.get(args.precision, M.FP32)
    ctx = M.Context(0)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", 0)
    measure_device(ctx, M, 0, stream)
    phs = [M.Phantom(ctx, [torch.from_numpy(a).to(dev) for a in w.phantom.arrays()], stream=stream) for w in ws]
    sqs = [M.Sequence.from_workload_sequence(ctx, w.sequence) for w in ws]
    outs = [torch.zeros(max(2 * q.n_adc, 2), dtype=torch.float64, device=dev) for q in sqs]
    b = M.Batch(ctx, phs, sqs, prec, outs)
    t0 = time.perf_counter()
    if args.spins_per_thread and args.threads:  # a fixed shape (profiling runs: no tuning launches)
        shape = (args.spins_per_thread, args.threads)
        b.set_shape(*shape)
    else:
        shape = b.autotune(stream=stream)
    tune_s = time.perf_counter() - t0
    spin_steps = sum(w.spin_steps for w in ws)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        b.launch(stream=stream, graph=True)
    ctx.stream_status(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.15)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush_buf.zero_()
        ev[i][0].record(stream)
        b.launch(stream=stream, graph=True)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ctx.stream_status(stream)
    ms = sum(a.elapsed_time(c) for a, c in ev) / args.steps
    kinds = [train_map_kinds(M, w.sequence.events, w.sequence.gamma_hz_per_t) for w in ws]
    form_ops = sum(map_adjusted(algorithmic_ops_per_spin(w.sequence.events), OPS_RF, km) * w.phantom.n
                   for w, km in zip(ws, kinds))
    ops = sum(map_adjusted(per_event_ops_per_spin(w.sequence.events, shape[0]), EV_RF, km) * w.phantom.n
              for w, km in zip(ws, kinds))
    achieved = ops / (ms * 1e-3) / 1e9
    form_g = form_ops / (ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": spin_steps / (ms * 1e-3), "unit": "spin-steps/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {M.FP64: "f64", M.FP32_KAHAN: "df32"}.get(prec, "f32"), "data": "synthetic",
        "config": {"workload": "c4_batch64", "n_phantoms": len(ws), "n_spins": sum(w.phantom.n for w in ws),
                   "spin_steps_per_step": spin_steps, "n_items": b.n_items,
                   "launch": {"spins_per_thread": shape[0], "threads_per_block": shape[1], "tune_s": tune_s,
                              "mode": "persistent kernel + work queue, CUDA graph replay"},
                   "l2": "flushed between timed steps (256 MB write, outside the step events)"},
        "roofline": fp64_roofline(achieved) if prec == M.FP64 else fp32_roofline(
            achieved, ck, traffic=traffic_for(kernel_source_sha(), "c4_batch64", program_sha(M, [w.sequence for w in ws])),
            kernel_ms=ms,
            ops_per_spin_step=ops / spin_steps,
            op_model=f"per event: ADC repeating the previous (G, dt) {EV_ADC_REPEAT}, RF {EV_RF}, other {EV_OTHER}, "
                     f"+ {EV_SAMPLE_TRANSPOSE}/k per sample with k = {shape[0]} spins per thread",
            formulation_model={"ops_per_spin_step": form_ops / spin_steps, "achieved": form_g,
                               "frac": form_g / (fp32_alu_peak_ops(sm_clock(ck)) / 1e9)}),
        # per step: the signal clear, every mapped phantom's train-map set-up, the batch kernel
        "gpu_launches": (2 + sum(1 for km in kinds if km)) * args.steps, "clocks": ck,
        "measured_rates": measured_rates(), "source": source_id(),
    }
    if prec == M.FP32 and not args.skip_extra:
        # the float64 and the compensated (double-float) batch on the same phantoms: their times,
        # and every phantom's float32 and compensated signal against the float64 one
        s32 = [o.clone() for o in outs]

        def other(pr, tune):
            o2 = [torch.zeros_like(o) for o in outs]
            b2 = M.Batch(ctx, phs, sqs, pr, o2)
            sh = b2.autotune(stream=stream) if tune else None
            b2.launch(stream=stream, graph=True)  # capture + first run
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b2.launch(stream=stream, graph=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ctx.stream_status(stream)
            t = e0.elapsed_time(e1)
            b2.close()
            return o2, t, sh

        s64, ms64, _ = other(M.FP64, False)
        sk, msk, shk = other(M.FP32_KAHAN, True)

        def per_phantom(got):
            errs = []
            for w, g, r in zip(ws, got, s64):
                a, b_ = g.cpu().numpy(), r.cpu().numpy()
                nb = float(np.linalg.norm(b_))
                errs.append((float(np.linalg.norm(a - b_) / nb) if nb > 0 else 0.0, w.name, w.sequence.name))
            errs.sort(reverse=True)
            return {"max": errs[0][0], "n_above_2e-5": sum(e > 2e-5 for e, _, _ in errs),
                    "max_flash": max((e for e, _, q in errs if q.startswith("flash")), default=0.0),
                    "max_spin_echo": max((e for e, _, q in errs if q.startswith("se")), default=0.0),
                    "worst": [[n, q, e] for e, n, q in errs[:6]]}

        line["fp64_gpu"] = {"value": spin_steps / (ms64 * 1e-3), "unit": "spin-steps/s", "ms_per_step": ms64,
                            "roofline": fp64_roofline(ops / (ms64 * 1e-3) / 1e9)}
        line["fp32_kahan_gpu"] = {"value": spin_steps / (msk * 1e-3), "unit": "spin-steps/s", "ms_per_step": msk,
                                  "launch": {"spins_per_thread": shk[0], "threads_per_block": shk[1]},
                                  "arithmetic": "double-float (float32 pairs with their rounding error) on the FP32 pipe"}
        line["per_phantom_vs_fp64_gpu"] = {"fp32": per_phantom(s32), "fp32_kahan": per_phantom(sk)}
    if not args.no_cpu_baseline:  # the oracle on a bounded spin sample of the batch's longest program
        wl = max(ws, key=lambda w: w.sequence.n_events)
        cb, (sub, ref) = cpu_baseline(wl, seconds=args.cpu_seconds)
        cb["sample"] = "c4 phantom " + cb["sample"]
        line["cpu_baseline"] = cb
        line["oracle_parity"] = dict(oracle_parity(ctx, M, wl, sub, ref), phantom=wl.name)
    print(json.dumps(line), flush=True)
    return 0


# Adjoint (float64) work per spin-step, in float64 flops (an FMA is 2): forward step = pulse
# (3x3 matrix-vector, 18 when the event has one) + precession/T2 (8) + T1 (3); the backward pass
# recomputes the forward step and applies the transposed step (pulse 18, its flip derivative 18 +
# 6 when the flip is learnable, precession 8, T1 3, parameter gradients 12).
ADJ_FLOPS_FWD_RF, ADJ_FLOPS_FWD = 18, 11
ADJ_FLOPS_BWD_RF, ADJ_FLOPS_BWD = 42, 23


def run_adjoint(args):
    """Differentiation workload (C5): one step = adjoint forward (signal + checkpoints) and backward
    (gradients in M0, T1, T2 of every spin and in the 256 learnable RF flips), float64."""
    import torch

    from paper_1305_6861_gb300 import mrsim as M

    torch.cuda.set_device(0)
    w, tgt, rf0 = W.config5()
    ev = w.sequence.events
    params = np.full(len(ev), -1, dtype=np.int32)
    idx = W.rf_event_index(w.sequence)
    params[idx] = np.tile(np.arange(len(rf0), dtype=np.int32), idx.size // len(rf0))
    ctx = M.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    measure_device(ctx, M, 0, stream)
    adj = M.Adjoint(ctx, ev, W.GAMMA_BAR, params, len(rf0), ckpt_every=64)
    kahan = args.precision == "kahan"
    if kahan:  # the recursion in double-float pairs on the FP32 pipe
        adj.set_precision(M.FP32_KAHAN)
    P = M.Phantom(ctx, [torch.from_numpy(a).to(dev) for a in w.phantom.arrays()], stream=stream)
    rfd = torch.from_numpy(rf0.copy()).to(dev)
    sig = torch.zeros(2 * adj.n_adc, dtype=torch.float64, device=dev)
    target = torch.zeros_like(sig)
    PT = M.Phantom(ctx, [torch.from_numpy(a).to(dev) for a in tgt.arrays()], stream=stream)
    adj.forward(PT, rfd, target, stream)
    grads = [torch.zeros(w.phantom.n, dtype=torch.float64, device=dev) for _ in range(3)]
    drf = torch.zeros(len(rf0), dtype=torch.float64, device=dev)

    def step():
        adj.forward(P, rfd, sig, stream)
        h = 2 * (sig - target)
        adj.backward(P, h, rfd, *grads, drf, stream)

    for _ in range(args.warmup):
        step()
    ctx.stream_status(stream)
    ev0 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.15)
    torch.cuda.synchronize()
    for i in range(args.steps):
        ev0[i][0].record(stream)
        step()
        ev0[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.stream_status(stream)
    ms = sum(a.elapsed_time(b) for a, b in ev0) / args.steps
    ck = clocks.stop()
    n_rf = int(np.count_nonzero(ev["rf_flip"] != 0))
    n_ev = len(ev)
    flops_spin = (2 * ADJ_FLOPS_FWD * n_ev + 2 * ADJ_FLOPS_FWD_RF * n_rf  # forward + recompute
                  + ADJ_FLOPS_BWD * n_ev + ADJ_FLOPS_BWD_RF * n_rf)
    flops = flops_spin * w.phantom.n
    achieved = flops / (ms * 1e-3) / 1e9
    fp64_peak = 2 * DEVICE["fp64_lane_ops_per_s"] / 1e9
    roof = {"bound": "fp64", "achieved": achieved, "peak": fp64_peak, "unit": "GFLOP/s (float64)",
            "frac": achieved / fp64_peak, "traffic": None, "kernel_ms": ms,
            "peak_basis": "2 x the float64 multiply-add rate measured on every SM in this run "
                          f"(SM clock {DEVICE['probe_sm_mhz']} MHz)",
            "flops_per_spin_step": flops_spin / n_ev}
    if kahan:  # the same arithmetic in double-float pairs, against the FP32 pipe
        roof = fp32_roofline(achieved / 2, ck, traffic=None, kernel_ms=ms, flops_per_spin_step=flops_spin / n_ev,
                             op_model="the float64 flop model's multiply-adds, executed as double-float pairs "
                                      "(each about 10-20 float32 operations)")
    line = {"metric": "spin-steps/s of forward+backward (adjoint) at 1 GB300", "value": w.spin_steps / (ms * 1e-3),
            "unit": "spin-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "df32" if kahan else "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "n_spins": w.phantom.n, "n_events": len(ev), "n_rf_params": len(rf0),
                       "ckpt_every": 64, "step": "adjoint forward + backward",
                       "note": "float64-pipe bound (ncu: the backward kernel keeps it 71 % busy with 4 warps per SM); the flop model counts the formulation's arithmetic, about half the executed float64 instructions"},
            "roofline": roof,
            "gpu_launches": 4 * args.steps, "clocks": ck, "measured_rates": measured_rates(), "source": source_id()}
    if not args.no_cpu_baseline:  # the oracle's forward-mode gradient (every flip) on a bounded spin sample
        import oracle

        cores = len(os.sched_getaffinity(0))
        rng = np.random.default_rng(1)
        h = np.ones(adj.n_adc, dtype=np.complex128)
        sel = np.arange(len(rf0), dtype=np.int32)

        def grad_time(n):
            sub = w.phantom.subset(np.sort(rng.choice(w.phantom.n, n, replace=False)))
            t0 = time.perf_counter()
            oracle.gradient(sub, ev, W.GAMMA_BAR, h, params, rf0, sel, n_threads=cores)
            return time.perf_counter() - t0

        per_spin = grad_time(cores) / cores
        n = int(max(cores, min(w.phantom.n, args.cpu_seconds / max(per_spin, 1e-9))))
        el = grad_time(n)
        line["cpu_baseline"] = {"value": n * n_ev / el, "unit": "spin-steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"forward-mode gradient (M0, T1, T2 and all {len(rf0)} flips) of {n} of "
                                          f"{w.phantom.n} spins over the full sequence, {el:.1f} s"}
    print(json.dumps(line), flush=True)
    return 0


# K-t formalism: algorithmic FP32 lane-ops per (ensemble, step, order index i >= 0): the pulse's
# three rows of Eq. 4.14 (10 each: one real-by-complex product and two complex products fused
# into the sums) and the relaxation / precession of a_i, a_-i (4 each) and b_i (2)
KT_OPS_PER_ORDER = 30 + 10


def run_kt(args):
    """K-t workload (§4.2): a fingerprinting-style dictionary, 65 536 ensembles over (T1, T2, B1,
    Δf) through an inversion + 1000-pulse train with one order of unbalanced gradient per TR,
    configuration orders up to K = 127, one sample per TR."""
    import torch

    from paper_1305_6861_gb300 import mrsim as M

    torch.cuda.set_device(0)
    rng = np.random.default_rng(W.SEED_BASE + 6)
    n_sets, n_tr, K = args.kt_sets, 1000, 127
    d = W.kt_dictionary(n_sets, rng)
    steps = W.kt_fingerprint_sequence(n_tr, rng)
    n_samples = int(np.count_nonzero(steps["sample"]))
    prec = M.FP64 if args.precision == "fp64" else M.FP32
    ctx = M.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    measure_device(ctx, M, 0, stream)
    par = [torch.from_numpy(a.copy()).to(dev) for a in (d.t1, d.t2, d.b1, d.df)]
    out = torch.zeros(n_sets * 2 * n_samples, dtype=torch.float64, device=dev)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        M.kt_simulate(ctx, par[0], par[1], steps, K, b1=par[2], df=par[3], precision=prec, stream=stream, out=out)

    for _ in range(args.warmup):
        step()
    ctx.stream_status(stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.15)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush_buf.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ctx.stream_status(stream)
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    ens_steps = n_sets * len(steps)
    ops = ens_steps * (K + 1) * KT_OPS_PER_ORDER
    achieved = ops / (ms * 1e-3) / 1e9
    line = {"metric": "ensemble-steps/s of the K-t formalism (configuration populations) at 1 GB300",
            "value": ens_steps / (ms * 1e-3), "unit": "ensemble-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == M.FP64 else "f32", "data": "synthetic",
            "config": {"workload": f"kt_fingerprint_{n_sets}x{len(steps)}_K{K}", "n_ensembles": n_sets,
                       "n_steps": len(steps), "max_order": K, "n_samples": n_samples,
                       "order_steps_per_step": ens_steps * (K + 1),
                       "l2": "flushed between timed steps (256 MB write, outside the step events)"},
            "roofline": dict(fp64_roofline(achieved), kernel_ms=ms, ops_per_order_step=KT_OPS_PER_ORDER)
            if prec == M.FP64 else
            fp32_roofline(achieved, ck,
                          traffic=traffic_for(kernel_source_sha(KT_SOURCES), f"kt_fingerprint_{n_sets}x{len(steps)}_K{K}"),
                          kernel_ms=ms, ops_per_order_step=KT_OPS_PER_ORDER),
            "gpu_launches": 2 * args.steps, "clocks": ck, "measured_rates": measured_rates(), "source": source_id()}
    if not args.no_cpu_baseline:
        from oracle import kt as ORK

        nb, t0, refs = 0, time.perf_counter(), []
        while time.perf_counter() - t0 < args.cpu_seconds and nb < n_sets:
            refs.append(ORK.simulate(d.t1[nb:nb + 1], d.t2[nb:nb + 1], d.b1[nb:nb + 1], d.df[nb:nb + 1], steps, K)[0])
            nb += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nb * len(steps) / dt, "unit": "ensemble-steps/s", "cores": 1, "kind": "oracle",
                                "sample": f"{nb} of {n_sets} ensembles, full train, {dt:.1f} s (numpy, one core)"}
        # the GPU's samples of those ensembles (last timed step) against the oracle's
        got = out.view(torch.complex128).view(n_sets, n_samples)[:nb].cpu().numpy()
        ref = np.stack(refs)
        rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        line["oracle_parity"] = {"sample_ensembles": nb, f"{'fp64' if prec == M.FP64 else 'fp32'}_rel_l2": rel,
                                 f"{'fp64' if prec == M.FP64 else 'fp32'}_db": 20 * math.log10(rel) if rel > 0 else None}
    print(json.dumps(line), flush=True)
    return 0


# Non-parallel fields: FP32 lane-operations per spin and event of the cached-map formulation.  An
# interval computed from its record (a new interval, or an anchored step of a run): the gradient
# field G.x (3), n.b (3), b - (n.b) n (3) and its square (3), u = B0 n + b (3), |u|^2 (3), the
# remainder r^2/(|u| + B0 + n.b) (2), h = u/|u| (3), the phase from four float-float products (6
# each) and its reduction (3), the map A = E2 cos(th) (I - h h^T) - E2 sin(th) [h]x + E1 h h^T and
# c = M0 (1 - E1) h (22) and its application (9): 81; with transverse components 6 more for
# (gtx.x, gty.x) and six more products (36).  An interval equal to the one whose map the spin
# holds: the map (9).  A pulse is the 3x3 rotation (9), a sample the demodulated value (4).
# Transcendentals (sin/cos, exp, square root, division) are not counted.
FIELD_OPS_COMPUTED, FIELD_OPS_TRANSVERSE, FIELD_OPS_MAP, FIELD_OPS_RF, FIELD_OPS_ADC = 81, 42, 9, 9, 4
FIELD_ANCHOR = 32  # every 32nd step of a run of equal intervals, and its last, is computed from the run's start


FIELD_TRAIN_MAX = 256  # longest train the fields kernels map


def field_train_maps(events, g_transverse):
    """The fields records' train maps: trains (two or more consecutive pulsed events without
    samples sharing one free interval, at most FIELD_TRAIN_MAX) keyed by interval and pulses; a
    key that occurs 4 times or more is a map kind (first 16 by first occurrence).  Returns
    (mapped, kinds): per event whether it belongs to a mapped train, and per kind (events,
    occurrences)."""
    n = len(events)
    gt = np.zeros((n, 6)) if g_transverse is None else np.asarray(g_transverse, dtype=float)
    key = np.concatenate([np.stack([events["dt"], events["gx"], events["gy"], events["gz"]], axis=1), gt], axis=1)
    pulsed = (events["rf_flip"] != 0) & (events["dt"] > 0) & (events["adc"] == 0)
    starts = {}
    i = 0
    while i < n:
        if not pulsed[i]:
            i += 1
            continue
        k = i + 1
        while k < n and k - i < FIELD_TRAIN_MAX and pulsed[k] and np.array_equal(key[k], key[i]):
            k += 1
        if k - i >= 2:
            tk = (tuple(key[i]), tuple(events["rf_flip"][i:k]), tuple(events["rf_phase"][i:k]))
            starts.setdefault(tk, []).append((i, k))
        i = k
    mapped = np.zeros(n, dtype=bool)
    kinds = []
    for occ in sorted(starts.values(), key=lambda v: v[0][0]):
        if len(kinds) == 16:
            break
        if len(occ) < 4:
            continue
        kinds.append((occ[0][1] - occ[0][0], len(occ)))
        for i0, k in occ:
            mapped[i0:k] = True
    return mapped, kinds


def field_event_classes(events, g_transverse, maps=True):
    """Which events compute their interval from the record (`computed`) and which apply the map the
    spin holds (`repeat`), as the field records mark them: a run is a sequence of equal free
    intervals (equal dt, G and transverse components) without pulses; its FIELD_ANCHOR-th steps
    and its last are computed from the run's start; any other interval equal to the last computed
    one (not counting anchored steps) repeats it.  With train maps, the events of mapped trains are
    neither (they run as their train's map) and leave the held map alone."""
    n = len(events)
    gt = np.zeros((n, 6)) if g_transverse is None else np.asarray(g_transverse, dtype=float)
    key = np.concatenate([np.stack([events["dt"], events["gx"], events["gy"], events["gz"]], axis=1), gt], axis=1)
    mapped = field_train_maps(events, g_transverse)[0] if maps else np.zeros(n, dtype=bool)
    free = events["dt"] > 0
    runnable = free & (events["rf_flip"] == 0)
    run = np.zeros(n, dtype=np.int64)
    for i in range(n):
        if runnable[i]:
            run[i] = run[i - 1] + 1 if i > 0 and run[i - 1] > 0 and np.array_equal(key[i], key[i - 1]) else 1
    length = np.zeros(n, dtype=np.int64)
    for i in range(n - 1, -1, -1):
        if run[i] > 0:
            length[i] = length[i + 1] if i + 1 < n and run[i + 1] == run[i] + 1 else run[i]
    anchor = (run > 1) & ((run % FIELD_ANCHOR == 0) | (run == length))
    computed = np.zeros(n, dtype=bool)
    repeat = np.zeros(n, dtype=bool)
    cached = None
    for i in range(n):
        if not free[i] or mapped[i]:
            continue
        if anchor[i]:
            computed[i] = True
        elif cached is not None and np.array_equal(key[i], cached):
            repeat[i] = True
        else:
            computed[i] = True
            cached = key[i]
    return computed, repeat


def field_ops_per_spin(events, g_transverse, maps=True) -> int:
    computed, repeat = field_event_classes(events, g_transverse, maps)
    mapped, kinds = field_train_maps(events, g_transverse) if maps else (np.zeros(len(events), dtype=bool), [])
    tr = np.any(g_transverse != 0, axis=1) if g_transverse is not None else np.zeros(len(events), dtype=bool)
    ops = (FIELD_OPS_COMPUTED * np.count_nonzero(computed) + FIELD_OPS_TRANSVERSE * np.count_nonzero(computed & tr)
           + FIELD_OPS_MAP * np.count_nonzero(repeat) + FIELD_OPS_RF * np.count_nonzero((events["rf_flip"] != 0) & ~mapped)
           + FIELD_OPS_ADC * np.count_nonzero(events["adc"]))
    # mapped trains: the map per occurrence; per kind, the interval's turn and four states stepped
    # through its events (pulse, then the turn)
    ops += sum(occ * EV_MAP + FIELD_OPS_COMPUTED + FIELD_OPS_TRANSVERSE + 4 * (FIELD_OPS_RF + FIELD_OPS_MAP) * n
               for n, occ in kinds)
    return int(ops)


def run_fields(args):
    """Non-parallel fields (static-field direction per spin, Maxwell concomitant gradient
    components): the 256² spin echo with a 10° smooth tilt at 1.5 T.  One step = one forward
    simulation of the whole phantom through mrsim_simulate_fields."""
    import torch

    from paper_1305_6861_gb300 import mrsim as M

    torch.cuda.set_device(0)
    w = W.config_fields(base="c2")
    prec = M.FP64 if args.precision == "fp64" else M.FP32
    ctx = M.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    measure_device(ctx, M, 0, stream)
    P = M.Phantom(ctx, [torch.from_numpy(a).to(dev) for a in w.phantom.arrays()], stream=stream)
    M.set_b0_direction(ctx, P, torch.from_numpy(w.b0_dir.reshape(-1).copy()).to(dev), stream=stream)
    F = M.Fields(ctx, w.sequence.events, W.GAMMA_BAR, w.g_transverse, w.b0_tesla)
    sig = torch.zeros(2 * F.n_adc, dtype=torch.float64, device=dev)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        M.simulate_fields(ctx, P, F, prec, stream=stream, out=sig)
    ctx.stream_status(stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.15)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush_buf.zero_()
        evs[i][0].record(stream)
        M.simulate_fields(ctx, P, F, prec, stream=stream, out=sig)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ctx.stream_status(stream)
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    ops = field_ops_per_spin(w.sequence.events, w.g_transverse) * w.phantom.n
    achieved = ops / (ms * 1e-3) / 1e9
    line = {"metric": "spin-steps/s of the non-parallel-field simulation at 1 GB300", "value": w.spin_steps / (ms * 1e-3),
            "unit": "spin-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == M.FP64 else "f32", "data": "synthetic",
            "config": {"workload": w.name, "n_spins": w.phantom.n, "n_events": w.sequence.n_events, "n_adc": F.n_adc,
                       "b0_tesla": w.b0_tesla, "max_tilt_deg": 10.0, "transverse": "Maxwell concomitant components",
                       "l2": "flushed between timed steps (256 MB write, outside the step events)"},
            "roofline": dict(fp64_roofline(achieved), kernel_ms=ms, ops_per_spin_step=ops / w.spin_steps)
            if prec == M.FP64 else fp32_roofline(achieved, ck, traffic=None, kernel_ms=ms,
                                                  ops_per_spin_step=ops / w.spin_steps,
                                                  op_model="cached-map formulation per event (a computed interval 81 (+42 "
                                                           "transverse), a repeated one 9, pulse 9, sample 4), "
                                                           "transcendentals not counted"),
            "gpu_launches": (2 if F.n_train_maps else 1) * args.steps, "clocks": ck, "measured_rates": measured_rates(),
            "source": source_id()}
    if not args.no_cpu_baseline:  # the oracle on a bounded spin sample, and the GPU on the same spins
        cb = cpu_baseline_fields(w, args.cpu_seconds)
        line["cpu_baseline"] = cb["baseline"]
        sub = cb["sample"]
        # the sample through the timed launch shape: the whole phantom with M0 = 0 outside it
        ps = M.Phantom.from_workload_phantom(ctx, masked_phantom(w.phantom, sub))
        M.set_b0_direction(ctx, ps, w.b0_dir)
        par = {"sample_spins": int(sub.size), "launch": "whole phantom, M0 = 0 outside the sample"}
        nr = float(np.linalg.norm(cb["ref"]))
        for name, pr in (("fp32", M.FP32), ("fp64", M.FP64)):
            got = M.simulate_fields(ctx, ps, F, pr)
            rel = float(np.linalg.norm(got - cb["ref"]) / nr)
            par[f"{name}_rel_l2"] = rel
            par[f"{name}_db"] = 20 * math.log10(rel) if rel > 0 else None
        line["oracle_parity"] = par
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_fields(w, seconds: float = 10.0, seed: int = 3):
    """CPU-baseline leg of the field workload: the oracle, as it stands, on a bounded spin sample
    (full sequence)."""
    import oracle

    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(seed)
    pool = np.nonzero(w.phantom.rho > 0)[0]

    def timed(idx):
        t0 = time.perf_counter()
        ref, _ = oracle.simulate_fields(w.phantom.subset(idx), w.sequence.events, W.GAMMA_BAR, w.b0_dir[idx],
                                        w.g_transverse, w.b0_tesla, n_threads=cores)
        return ref, time.perf_counter() - t0

    cal = np.sort(rng.choice(pool, min(cores * 4, pool.size), replace=False))
    _, dt = timed(cal)
    n = int(max(cores, min(pool.size, seconds / max(dt / cal.size, 1e-9))))
    idx = np.sort(rng.choice(pool, n, replace=False))
    ref, el = timed(idx)
    return {"baseline": {"value": n * w.sequence.n_events / el, "unit": "spin-steps/s", "cores": cores,
                         "kind": "oracle", "sample": f"{w.name}: full sequence ({w.sequence.n_events} events) on "
                                                     f"{n} of {w.phantom.n} spins, {el:.1f} s"},
            "sample": idx, "ref": ref}


def run_ours(args):
    import torch

    from paper_1305_6861_gb300 import mrsim as M

    if args.workload == "c4":
        return run_batch(args)
    if args.workload == "c5":
        return run_adjoint(args)
    if args.workload == "kt":
        return run_kt(args)
    if args.workload == "fields":
        return run_fields(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    w = build_workload(args.workload, rank)
    canonical = w.sequence
    if args.raster:
        if args.events:
            raise SystemExit("--raster and --events do not combine")
        w = rasterized(w, args.raster)
    if args.events:  # profiling aid: a prefix of the sequence (whole repetitions), named in config
        w = W.Workload(w.name + f"_first{args.events}ev", w.phantom,
                       W.Sequence(w.sequence.events[: args.events], w.sequence.gamma_hz_per_t), w.note)
    prec = {"fp64": M.FP64, "kahan": M.FP32_KAHAN}.get(args.precision, M.FP32)
    ctx = M.Context(local)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)
    measure_device(ctx, M, local, stream)
    arrs = [torch.from_numpy(a).to(dev) for a in w.phantom.arrays()]
    ph = M.Phantom(ctx, arrs, stream=stream)
    seq = M.Sequence.from_workload_sequence(ctx, w.sequence)
    n_coils = args.coils
    sig = torch.zeros(2 * seq.n_adc * max(n_coils, 1), dtype=torch.float64, device=dev)
    sens_dev = None
    if n_coils:
        sens_dev = torch.from_numpy(ring_coils(w.phantom, n_coils).view(np.float64).reshape(-1).copy()).to(dev)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    kw = {}
    if args.spins_per_thread:
        kw["spins_per_thread"] = args.spins_per_thread
    if args.threads:
        kw["threads_per_block"] = args.threads
    tuned = None
    if not kw and not args.no_tune and not n_coils:  # autotune the launch shape (part of warm-up, outside the timed region)
        t0 = time.perf_counter()
        tuned = M.autotune(ctx, ph, seq, prec, stream=stream)
        tuned = {"spins_per_thread": tuned[0], "threads_per_block": tuned[1], "tune_s": time.perf_counter() - t0}
    if n_coils:
        k_spins = 2 if prec == M.FP32 else 1  # the coil kernels' fixed spins per thread
    else:
        k_spins = kw.get("spins_per_thread") or (tuned or {}).get("spins_per_thread") or 8
    # the launch shape of the timed runs (0, 0: the library's choice)
    shape = (kw.get("spins_per_thread") or (tuned or {}).get("spins_per_thread") or 0,
             kw.get("threads_per_block") or (tuned or {}).get("threads_per_block") or 0)

    def simulate_once():
        if n_coils:
            M.simulate_coils(ctx, ph, seq, sens_dev, prec, stream=stream, out=sig)
        else:
            M.simulate(ctx, ph, seq, prec, stream=stream, out=sig, **kw)

    def step():
        simulate_once()
        D.reduce_signal(sig)

    for _ in range(args.warmup):
        step()
    ctx.stream_status(stream)

    # the float64 oracle on a spin sample runs on the host cores meanwhile (rank 0, plain lists)
    # (one GPU only: a multi-GPU run holds every GPU while rank 0 would run them)
    extras = world == 1 and not args.skip_extra and not n_coils and prec != M.FP32_KAHAN
    frac = args.oracle_fraction if args.oracle_fraction >= 0 else {"c1": 1.0, "c2": 1.0, "c3": 0.01}[args.workload]
    orun = None
    if extras and not args.no_cpu_baseline and not args.raster and not args.events and frac > 0:
        orun = cpu_baseline_parity_run(w, sample_index(w.phantom, frac))

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.15)
    barrier()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush_buf.zero_()  # L2 flush between timed steps (outside the step's events)
        ev[i][0].record(stream)
        kev[i][0].record(stream)
        simulate_once()
        kev[i][1].record(stream)
        D.reduce_signal(sig)
        ev[i][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    ck = clocks.stop()
    ctx.stream_status(stream)
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    kern_ms = sum(a.elapsed_time(b) for a, b in kev) / args.steps
    ms_per_step = D.max_over_ranks(step_ms, device=dev) / args.steps
    spin_steps = w.spin_steps
    value = world * spin_steps / (ms_per_step * 1e-3)

    # ---- roofline of the dominant kernel (the forward kernel; one launch per step) ----------
    base_ev = (canonical if args.raster else w.sequence).events
    # recurring shaped pulses run as train maps
    kinds = train_map_kinds(M, base_ev, w.sequence.gamma_hz_per_t)
    form_ops = map_adjusted(algorithmic_ops_per_spin(base_ev, n_coils), OPS_RF, kinds) * w.phantom.n
    form_g = form_ops / (kern_ms * 1e-3) / 1e9
    sha = kernel_source_sha()
    map_note = (f"; {sum(o for _, o in kinds)} recurring trains of {len(kinds)} kinds as maps: {EV_MAP} per "
                f"occurrence instead of its sub-pulses, 4 x RF per sub-pulse per kind to form them") if kinds else ""
    if n_coils:  # the per-event model has no coil term: the formulation model is the algorithmic work
        ops, model = form_ops, "formulation model with receive coils (a sample costs 4 + 4 per coil)" + map_note
    else:
        ops = map_adjusted(per_event_ops_per_spin(base_ev, k_spins), EV_RF, kinds) * w.phantom.n
        model = (f"per event: ADC repeating the previous (G, dt) {EV_ADC_REPEAT}, RF {EV_RF}, other {EV_OTHER}, "
                 f"+ {EV_SAMPLE_TRANSPOSE}/k per sample with k = {k_spins} spins per thread" + map_note)
    achieved = ops / (kern_ms * 1e-3) / 1e9
    if prec == M.FP64:  # the same algorithmic lane-ops against the measured float64 rate
        roof = dict(fp64_roofline(achieved), kernel_ms=kern_ms, ops_per_spin_step=ops / spin_steps, op_model=model)
    else:
        roof = fp32_roofline(
            achieved, ck, traffic=traffic_for(sha, w.name + (f"_{n_coils}coils" if n_coils else ""),
                                              program_sha(M, [w.sequence])),
            kernel_ms=kern_ms, ops_per_spin_step=ops / spin_steps, op_model=model,
            formulation_model={"ops_per_spin_step": form_ops / spin_steps, "achieved": form_g,
                               "frac": form_g / (fp32_alu_peak_ops(sm_clock(ck)) / 1e9),
                               "basis": f"ADC {OPS_ADC}, RF {OPS_RF}, other {OPS_OTHER} (pulse-frame formulation)"})

    out = {}
    if extras:
        # float64 GPU path on the same workload, and its agreement with float32
        s32 = sig.clone()
        if dist:
            M.simulate(ctx, ph, seq, M.FP32, stream=stream, out=s32, **kw)
        other = M.FP32 if prec == M.FP64 else M.FP64
        so = torch.zeros_like(sig)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if kern_ms < 200.0:  # short kernels: one untimed run, then two timed ones
            M.simulate(ctx, ph, seq, other, stream=stream, out=so)
            reps = 2
        else:  # a long kernel is timed on its one run (launch overheads are negligible)
            reps = 1
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            M.simulate(ctx, ph, seq, other, stream=stream, out=so)
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.stream_status(stream)
        o_ms = e0.elapsed_time(e1) / reps
        a32 = (s32 if prec == M.FP32 else so).cpu().numpy().view(np.complex128)
        a64 = (so if prec == M.FP32 else s32).cpu().numpy().view(np.complex128)
        rel = float(np.linalg.norm(a32 - a64) / np.linalg.norm(a64))
        key = "fp64_gpu" if prec == M.FP32 else "fp32_gpu"
        out[key] = {"value": spin_steps / (o_ms * 1e-3), "unit": "spin-steps/s", "ms_per_step": o_ms, "runs": reps}
        if key == "fp64_gpu":  # the same algorithmic lane-ops against the measured float64 rate
            out[key]["roofline"] = fp64_roofline(ops / (o_ms * 1e-3) / 1e9)
        out["fp32_vs_fp64_gpu_rel_l2"] = rel
        out["fp32_vs_fp64_gpu_db"] = 20 * math.log10(rel) if rel > 0 else None
        if not args.no_kahan and prec == M.FP32:
            # the compensated precision (double-float on the FP32 pipe): one timed run and its
            # agreement with the float64 path
            sk = torch.zeros_like(sig)
            kk = M.autotune(ctx, ph, seq, M.FP32_KAHAN, stream=stream)
            M.simulate(ctx, ph, seq, M.FP32_KAHAN, stream=stream, out=sk)  # warm-up
            torch.cuda.synchronize()
            e0.record(stream)
            M.simulate(ctx, ph, seq, M.FP32_KAHAN, stream=stream, out=sk)
            e1.record(stream)
            torch.cuda.synchronize()
            ctx.stream_status(stream)
            k_ms = e0.elapsed_time(e1)
            ak = sk.cpu().numpy().view(np.complex128)
            rk = float(np.linalg.norm(ak - a64) / np.linalg.norm(a64))
            out["fp32_kahan_gpu"] = {"value": spin_steps / (k_ms * 1e-3), "unit": "spin-steps/s", "ms_per_step": k_ms,
                                     "launch": {"spins_per_thread": kk[0], "threads_per_block": kk[1]},
                                     "rel_l2_vs_fp64_gpu": rk,
                                     "arithmetic": "double-float (float32 pairs with their rounding error) on the FP32 pipe"}
        if orun is not None:
            out["oracle_parity"] = oracle_parity_sample(ctx, M, w, orun, seq, shape, stream)

        if not args.no_cpu_baseline:  # the oracle alone on the host cores, on a bounded sample
            cb, (sub, ref) = cpu_baseline(w, seconds=args.cpu_seconds)
            out["cpu_baseline"] = cb
            if orun is None:
                out["oracle_parity"] = oracle_parity(ctx, M, w, sub, ref)
    # end to end through the public API with host buffers (pinned), copies inside the region; with
    # more than one GPU every rank runs it on its own spins and the signal is summed across ranks
    # in every step, as in the timed steps
    if not args.skip_extra and not n_coils and prec != M.FP32_KAHAN:
        pinned = [torch.from_numpy(a).pin_memory() for a in w.phantom.arrays()]
        host_arrays = [p.numpy() for p in pinned]
        ev_pinned = torch.from_numpy(w.sequence.events.view(np.uint8)).pin_memory().numpy().view(W.EVENT_DTYPE)
        host_sig = torch.zeros(2 * seq.n_adc, dtype=torch.float64).pin_memory()
        host_sig_c = host_sig.numpy().view(np.complex128)
        dev_sig = torch.zeros(2 * seq.n_adc, dtype=torch.float64, device=dev)
        e2e_steps = max(3, min(args.steps, 20))
        serial_steps = e2e_steps if kern_ms < 200.0 else 3
        gamma = w.sequence.gamma_hz_per_t

        def run_e2e(p, s):
            if dist:  # device output, the sum over ranks, then the read-back
                M.simulate(ctx, p, s, prec, stream=stream, out=dev_sig, **kw)
                D.reduce_signal(dev_sig)
                host_sig.copy_(dev_sig)
            else:
                M.simulate(ctx, p, s, prec, out=host_sig_c, **kw)

        def e2e_serial_step():
            p = M.Phantom(ctx, host_arrays)
            s = M.Sequence(ctx, ev_pinned, gamma)
            run_e2e(p, s)
            p.close()
            s.close()

        def e2e_pipelined(n):
            # each step: host compile (mrsim_compile, no context: on a worker thread, one step
            # ahead), phantom upload, program upload, simulation, signal read-back
            from concurrent.futures import ThreadPoolExecutor

            with ThreadPoolExecutor(1) as pool:
                nxt = pool.submit(M.Compiled, ev_pinned, gamma)
                for i in range(n):
                    comp = nxt.result()
                    if i + 1 < n:
                        nxt = pool.submit(M.Compiled, ev_pinned, gamma)
                    p = M.Phantom(ctx, host_arrays)
                    s = M.Sequence.from_compiled(ctx, comp)
                    comp.close()
                    run_e2e(p, s)
                    p.close()
                    s.close()

        e2e_serial_step()
        e2e_pipelined(2)
        torch.cuda.synchronize()
        serial_s = None
        if not dist:
            t0 = time.perf_counter()
            for _ in range(serial_steps):
                e2e_serial_step()
            torch.cuda.synchronize()
            serial_s = (time.perf_counter() - t0) / serial_steps
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_pipelined(e2e_steps)
        torch.cuda.synchronize()
        e2e_s = D.max_over_ranks((time.perf_counter() - t0) * 1e3, device=dev) / 1e3 / e2e_steps
        upload = M.Compiled(ev_pinned, gamma)
        h2d = int(7 * 8 * w.phantom.n + upload.upload_bytes)
        upload.close()
        out["e2e"] = {"value": world * spin_steps / e2e_s, "unit": "spin-steps/s", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": int(16 * seq.n_adc), "ms_per_step": e2e_s * 1e3, "steps": e2e_steps,
                      "pipeline": "the next step's host compile runs on a worker thread during this step's "
                                  "uploads, kernel and read-back (first compile not overlapped)"
                                  + ("; per step the signal is summed across ranks before the read-back; slowest rank"
                                     if dist else "")}
        if serial_s is not None:
            out["e2e"].update({"serial_ms_per_step": serial_s * 1e3, "serial_steps": serial_steps})
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "spin-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {M.FP64: "f64", M.FP32_KAHAN: "df32"}.get(prec, "f32"), "data": "synthetic",
            "config": {"workload": w.name + (f"_{n_coils}coils" if n_coils else ""), "n_spins_per_gpu": w.phantom.n,
                       "n_events": w.sequence.n_events,
                       "n_adc": seq.n_adc, "n_ops": seq.n_ops, "spin_steps_per_gpu_step": spin_steps,
                       "precision": args.precision, "launch": kw or tuned or "library default",
                       "l2": "flushed between timed steps (256 MB write, outside the step events)",
                       "parallelism": f"spin-sharded x{world}" if world > 1 else "1 GPU",
                       **({"stress_mode": RASTER_NOTE.format(r=args.raster * 1e6, n=canonical.n_events)}
                          if args.raster else {})},
            "roofline": roof, "gpu_launches": (2 if kinds else 1) * args.steps, "clocks": ck, "wall_s_timed": t_wall,
            "measured_rates": measured_rates(),
            "peaks_file": {k: read_peaks().get(k) for k in ("hbm_gbs", "bf16_tflops", "sm_max_mhz")},
            "source": source_id(),
        }
        line.update(out)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["c1", "c2", "c3", "c4", "c5", "kt", "fields"], default="c3")
    ap.add_argument("--kt-sets", type=int, default=65536, help="ensembles of the K-t workload")
    ap.add_argument("--precision", choices=["fp32", "fp64", "kahan"], default="fp32",
                    help="kahan: the compensated precision (double-float on the FP32 pipe)")
    ap.add_argument("--spins-per-thread", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--oracle-fraction", type=float, default=-1.0,
                    help="oracle-parity sample as a fraction of the spin count, drawn from spins with M0 > 0 "
                         "(default: c1, c2 all spins; c3 1 %%)")
    ap.add_argument("--ref-seconds", type=float, default=5.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-extra", action="store_true")
    ap.add_argument("--no-kahan", action="store_true", help="skip the compensated-precision leg")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--events", type=int, default=0, help="use only the first N events (profiling cases)")
    ap.add_argument("--coils", type=int, default=0, help="receive coils (ring sensitivities), 0 = plain signal")
    ap.add_argument("--raster", type=float, default=0.0,
                    help="stress mode (c1-c3): cut every event into pieces of at most this many seconds (1e-5)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
