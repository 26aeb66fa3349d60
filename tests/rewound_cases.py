"""Sequences around the compiler's rewound-readout fold (a one-off precession A, a sample run R and
a one-off precession B whose moments add up to one that recurs; the run then starts with A and its
anchor covers A+R+B).  Test infrastructure: shared by the host-compiler and the GPU parity tests.

gamma = 1 Hz/T and durations that are powers of two make every moment γ·G·Δt exact in binary,
so that the sums the compiler forms are exact and the cases below are decided by structure alone.
"""
import math

import numpy as np

from paper_1305_6861_gb300 import workloads as W

GAMMA = 1.0
DT = 2.0**-10  # s
DWELL = 2.0**-14  # s


def _row(dt, gx=0.0, gy=0.0, gz=0.0, flip=0.0, phase=0.0, adc=0, adc_phase=0.0):
    return (dt, gx, gy, gz, flip, phase, adc, adc_phase)


def _readout(rows, n, g):
    for _ in range(n):
        rows.append(_row(DWELL, gx=g, adc=1, adc_phase=0.3))


def multi_echo(n_tr: int = 12, n_read: int = 16):
    """Per TR: pulse, A = (kx_pre, ky_m), R1, B, R2, C.  Both A+R1+B and B+R2+C recur, so the
    triples overlap at B: only the first may fold (B is its B), the second stays as it is."""
    rows = []
    g_read = 2048.0  # moment per sample 0.125 cycles/m
    for m in range(n_tr):
        ky = (m - n_tr // 2) * 1024.0  # moment ky·DT = (m - n/2) cycles/m
        rows.append(_row(DT, flip=0.4, phase=0.7 * m * m))
        rows.append(_row(DT, gx=-1024.0, gy=ky))  # A
        _readout(rows, n_read, g_read)  # R1
        rows.append(_row(DT, gx=-2048.0, gy=-ky + 512.0))  # B: A+R1+B = (-1, 0.5) cycles/m
        _readout(rows, n_read, g_read)  # R2
        rows.append(_row(DT, gx=512.0, gy=ky - 512.0))  # C: B+R2+C = (0.5, 0) cycles/m
        rows.append(_row(4 * DT))
    return W.make_events(rows)


def flash_like(n_tr: int = 16, n_read: int = 16, rewind: bool = True, jitter=None):
    """Gradient echo with phase encoding: A = (kx_pre, ky_m, kz), R, B = (spoil, -ky_m, -kz) (the
    fold applies); with `jitter` the rewinder misses -ky_m by a random amount (no recurrence, no
    fold); without `rewind` there is no B at all."""
    rows = []
    for m in range(n_tr):
        ky = (m - n_tr // 2) * 1024.0
        kz = ((m * 5) % 4 - 2) * 512.0
        rows.append(_row(DT, flip=0.5, phase=0.1 * m * (m + 1) / 2))
        rows.append(_row(DT, gx=-1024.0, gy=ky, gz=kz))
        _readout(rows, n_read, 2048.0)
        if rewind:
            e = 0.0 if jitter is None else float(jitter.uniform(-200.0, 200.0))
            rows.append(_row(2 * DT, gx=4096.0, gy=-ky / 2 + e, gz=-kz / 2))
        rows.append(_row(3 * DT))
    return W.make_events(rows)


def phantom(n: int, rng):
    ph = W.random_phantom(n, rng)
    return W.Phantom(ph.x * 0.4, ph.y * 0.4, ph.z * 0.4, ph.rho, ph.t1, ph.t2, ph.dw * 0.05)


def fold_counts(M, events, snapshots=None):
    """(folded runs, runs, inline precession ops) of the compiled program."""
    ops = M.debug_compile(events, GAMMA, snapshots=snapshots)["ops"]
    runs = ops[ops["kind"] == M.OP_RUN]
    folded = int(np.count_nonzero(runs["flags"] & M.F_INLINE))
    inline = int(np.count_nonzero((ops["kind"] == M.OP_PREC) & ((ops["flags"] & M.F_INLINE) != 0)))
    return folded, len(runs), inline


def phase_floor(ph, ev, gamma=GAMMA):
    g = 2 * math.pi * gamma
    th = (g * (np.abs(ev["gx"]) * np.abs(ph.x).max() + np.abs(ev["gy"]) * np.abs(ph.y).max()
               + np.abs(ev["gz"]) * np.abs(ph.z).max()) + np.abs(ph.dw).max()) * ev["dt"]
    return max(1e-12, 4 * 2.0**-53 * float(np.sqrt(np.sum(th**2))))
