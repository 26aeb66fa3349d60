"""K-t formalism oracle (§4.2): configuration populations of spin ensembles, plain numpy, float64.

TEST INFRASTRUCTURE ONLY: the correctness reference for the library's K-t kernel.  Only the
tests, the smoke check and the benchmark's CPU leg may use it.  It shares nothing with the CUDA
path.

An ensemble (one voxel's isochromats, or one entry of a parameter dictionary) is described by
the populations a_i of its transverse configurations E_i (i = -K..K) and b_i of its longitudinal
configurations Z_i (§4.2.1), M0 = 1, starting in thermal equilibrium (b_0 = 1).  One step is one
elementary sequence (Eq. 4.1):
  1. the hard pulse (flip B1·alpha, phase phi) mixes (a_i, a*_-i, b_i) with T'_HF of Eq. 4.2, for
     every order i (Eq. 4.14);
  2. over the interval tau: the gradient moves every transverse order by `shift` (Eq. 4.17:
     E_{±i} -> E_{±i+q}; populations pushed beyond ±K are dropped, the truncation of the K-t
     tree), relaxation scales a_i by E2 and b_i by E1 and adds (1 - E1) to b_0 (Eqs. 4.15, 4.16),
     and an off-resonance df turns every transverse population by exp(-j 2π df tau) (the ensemble's
     common precession, Eq. 3.14);
  3. a sampled step records a_0 (the ensemble's transverse magnetisation), demodulated by
     exp(-j adc_phase).
Reading: b_{-i} = conj(b_i), so that M_z = Z_0 is real (§4.2.2 states the symmetry of the
longitudinal configurations; the conjugate form is the one under which Eq. 4.14 maps the
populations of order -i consistently with those of order i).
"""
from __future__ import annotations

import math

import numpy as np

STEP_DTYPE = np.dtype([("alpha", "<f8"), ("phi", "<f8"), ("tau", "<f8"), ("adc_phase", "<f8"),
                       ("shift", "<i4"), ("sample", "<i4"), ("reserved", "<i8")])


def rf_matrix(alpha: float, phi: float) -> np.ndarray:
    """T'_HF of Eq. 4.2 acting on (M_xy, M*_xy, M_z)."""
    c2, s2, sa = math.cos(alpha / 2) ** 2, math.sin(alpha / 2) ** 2, math.sin(alpha)
    return np.array([
        [c2, s2 * np.exp(2j * phi), sa * np.exp(1j * (phi + math.pi / 2))],
        [s2 * np.exp(-2j * phi), c2, sa * np.exp(-1j * (phi + math.pi / 2))],
        [sa / 2 * np.exp(-1j * (phi - math.pi / 2)), sa / 2 * np.exp(1j * (phi - math.pi / 2)), math.cos(alpha)],
    ])


def simulate_one(t1: float, t2: float, b1: float, df: float, steps: np.ndarray, max_order: int) -> np.ndarray:
    """Signal (one complex value per sampled step) of one ensemble."""
    K = int(max_order)
    a = np.zeros(2 * K + 1, dtype=complex)  # a[K + i] = a_i
    b = np.zeros(2 * K + 1, dtype=complex)  # b[K + i] = b_i
    b[K] = 1.0
    out = []
    for st in steps:
        T = rf_matrix(b1 * float(st["alpha"]), float(st["phi"]))
        ac = np.conj(a[::-1])  # at index K + i: conj(a_-i)
        a, b = (T[0, 0] * a + T[0, 1] * ac + T[0, 2] * b,
                T[2, 0] * a + T[2, 1] * ac + T[2, 2] * b)
        q = int(st["shift"])
        if abs(q) >= a.size:  # every population leaves the kept orders
            a = np.zeros_like(a)
        elif q > 0:
            a = np.concatenate([np.zeros(q, dtype=complex), a[:-q]])
        elif q < 0:
            a = np.concatenate([a[-q:], np.zeros(-q, dtype=complex)])
        tau = float(st["tau"])
        e1 = math.exp(-tau / t1) if math.isfinite(t1) else 1.0
        e2 = math.exp(-tau / t2) if math.isfinite(t2) else 1.0
        a = a * e2 * np.exp(-2j * math.pi * df * tau)
        b = b * e1
        b[K] += 1.0 - e1
        if st["sample"]:
            out.append(a[K] * np.exp(-1j * float(st["adc_phase"])))
    return np.array(out, dtype=complex)


def simulate(t1, t2, b1, df, steps, max_order: int) -> np.ndarray:
    """Signals of n ensembles: complex [n, n_samples].  b1 / df may be None (1 / 0)."""
    t1 = np.asarray(t1, dtype=float)
    n = t1.shape[0]
    t2 = np.asarray(t2, dtype=float)
    b1 = np.ones(n) if b1 is None else np.asarray(b1, dtype=float)
    df = np.zeros(n) if df is None else np.asarray(df, dtype=float)
    for f in ("alpha", "phi", "tau", "adc_phase", "shift", "sample"):
        if f not in steps.dtype.names:
            raise ValueError(f"steps need field {f}")
    return np.stack([simulate_one(t1[s], t2[s], b1[s], df[s], steps, max_order) for s in range(n)])


def make_steps(rows) -> np.ndarray:
    """Rows of (alpha, phi, tau, shift, sample, adc_phase) → STEP_DTYPE array."""
    out = np.zeros(len(rows), dtype=STEP_DTYPE)
    for k, (al, ph, tau, q, smp, adc) in enumerate(rows):
        out[k] = (al, ph, tau, adc, q, smp, 0)
    return out
