"""Seeded synthetic inputs: phantoms (spin lists) and pulse sequences (event lists).

This module only *builds inputs*.  It holds none of the simulation arithmetic
(no rotation, precession, relaxation or signal sum): the CPU oracle under
``oracle/`` and the CUDA library both consume what it returns.

Object model (§6.1.1): every spin (isochromat) has a position, an equilibrium
magnetisation M0 (``rho``), relaxation times T1/T2 and a total off-resonance
angular frequency Δω (Eq. 6.2, rotating frame).  Several isochromats per voxel
share the voxel's M0 equally (M0_s = ρ_voxel / n_iso).

Sequence model (§4.1): a sequence is a list of elementary sequences ("events").
Each event has a duration Δt ≥ 0, a hard RF pulse (flip α, phase φ) acting at
its start, a constant gradient G = (Gx, Gy, Gz) for Δt, and optionally one ADC
sample taken at its end (§5.1.1: acquisition intervals are split into one step
per sample, the magnetisation is stored after each step).  ``adc_phase`` is the
receiver demodulation phase used with RF spoiling (an extension the paper does
not have; 0 everywhere else).

All generators draw from ``numpy.random.Generator(PCG64(seed))`` with
``seed = 13050000 + config_id`` by default.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# γ/2π for protons as printed in §3.2 (footnote): γ = 2π·42.6e6 1/(s·T).
GAMMA_BAR = 42.6e6

# One event record: 7 float64 + int32 adc flag + int32 reserved = 64 bytes.
EVENT_DTYPE = np.dtype(
    [
        ("dt", "<f8"),
        ("gx", "<f8"),
        ("gy", "<f8"),
        ("gz", "<f8"),
        ("rf_flip", "<f8"),
        ("rf_phase", "<f8"),
        ("adc_phase", "<f8"),
        ("adc", "<i4"),
        ("reserved", "<i4"),
    ],
    align=False,
)
assert EVENT_DTYPE.itemsize == 64

# (T1 [s], T2 [s], ρ) of the four 2D tissue classes.
TISSUES_2D = ((0.3, 0.04, 0.7), (0.8, 0.08, 0.8), (1.2, 0.1, 0.9), (4.0, 2.0, 1.0))
# Fat isochromats: chemical shift −3.5 ppm at 1.5 T → −223.65 Hz; T1/T2 (0.26, 0.08) s.
FAT_SHIFT_HZ = -3.5e-6 * GAMMA_BAR * 1.5
FAT_T1T2 = (0.26, 0.08)

SEED_BASE = 13050000


def rng_for(config_id: int, seed: int | None = None) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_id if seed is None else seed))


# ---------------------------------------------------------------------------
# Containers
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Phantom:
    """Spin list, SoA, float64, SI units (m, s, rad/s)."""

    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    rho: np.ndarray
    t1: np.ndarray
    t2: np.ndarray
    dw: np.ndarray

    def __post_init__(self):
        for f in dataclasses.fields(self):
            a = np.ascontiguousarray(getattr(self, f.name), dtype=np.float64)
            setattr(self, f.name, a)
        n = self.x.shape[0]
        for f in dataclasses.fields(self):
            if getattr(self, f.name).shape != (n,):
                raise ValueError(f"phantom field {f.name} has shape {getattr(self, f.name).shape}, expected ({n},)")

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def arrays(self):
        return (self.x, self.y, self.z, self.rho, self.t1, self.t2, self.dw)

    def subset(self, idx) -> "Phantom":
        return Phantom(*(a[idx] for a in self.arrays()))

    def concat(self, other: "Phantom") -> "Phantom":
        return Phantom(*(np.concatenate([a, b]) for a, b in zip(self.arrays(), other.arrays())))


@dataclasses.dataclass
class Sequence:
    events: np.ndarray  # EVENT_DTYPE
    gamma_hz_per_t: float = GAMMA_BAR
    kshape: tuple = ()  # k-space layout of the ADC samples, for reshaping only
    name: str = ""

    def __post_init__(self):
        self.events = np.ascontiguousarray(self.events, dtype=EVENT_DTYPE)

    @property
    def n_events(self) -> int:
        return int(self.events.shape[0])

    @property
    def n_adc(self) -> int:
        return int(np.count_nonzero(self.events["adc"]))


@dataclasses.dataclass
class Workload:
    name: str
    phantom: Phantom
    sequence: Sequence
    note: str = ""

    @property
    def spin_steps(self) -> int:
        return self.phantom.n * self.sequence.n_events


class _Events:
    """Append-only event list builder."""

    def __init__(self):
        self.rows = []

    def add(self, dt, gx=0.0, gy=0.0, gz=0.0, flip=0.0, phase=0.0, adc=0, adc_phase=0.0):
        if dt < 0:
            raise ValueError(f"negative event duration {dt}")
        self.rows.append((dt, gx, gy, gz, flip, phase, adc_phase, int(adc), 0))

    def array(self) -> np.ndarray:
        return np.array(self.rows, dtype=EVENT_DTYPE)


def make_events(rows) -> np.ndarray:
    """Rows of (dt, gx, gy, gz, flip, phase, adc, adc_phase) → EVENT_DTYPE array."""
    ev = _Events()
    for r in rows:
        ev.add(*r)
    return ev.array()


# ---------------------------------------------------------------------------
# Phantoms
# ---------------------------------------------------------------------------


def grid_coords(n: int, fov: float) -> np.ndarray:
    """Voxel-centre coordinates x_i = (i − n/2)·fov/n (the grid the imaging equation samples)."""
    return (np.arange(n) - n // 2) * (fov / n)


def _nested_ellipses(rng: np.random.Generator, levels: int = 4):
    """Random nested ellipses in normalised coordinates (FOV = 1): (cx, cy, ax, ay, angle)."""
    out = []
    cx, cy = rng.uniform(-0.04, 0.04, size=2)
    ax, ay = rng.uniform(0.34, 0.44, size=2)
    ang = rng.uniform(0, math.pi)
    out.append((cx, cy, ax, ay, ang))
    for _ in range(levels - 1):
        s = rng.uniform(0.5, 0.72)
        ax2, ay2 = ax * s, ay * s
        # shift inside the parent by at most a fraction of the spare room
        room = min(ax - ax2, ay - ay2) * 0.5
        cx, cy = cx + rng.uniform(-room, room), cy + rng.uniform(-room, room)
        ax, ay = ax2, ay2
        ang = rng.uniform(0, math.pi)
        out.append((cx, cy, ax, ay, ang))
    return out


def _ellipse_labels(ellipses, u, v) -> np.ndarray:
    """Deepest nested ellipse containing (u, v) (normalised coords); −1 outside all."""
    lab = np.full(u.shape, -1, dtype=np.int32)
    for i, (cx, cy, ax, ay, ang) in enumerate(ellipses):
        c, s = math.cos(ang), math.sin(ang)
        du, dv = u - cx, v - cy
        p = (c * du + s * dv) / ax
        q = (-s * du + c * dv) / ay
        lab[p * p + q * q <= 1.0] = i
    return lab


def _tissue_params(labels: np.ndarray, tissues=TISSUES_2D):
    t1 = np.ones(labels.shape)
    t2 = np.full(labels.shape, 0.1)
    rho = np.zeros(labels.shape)
    for i, (a, b, r) in enumerate(tissues):
        m = labels == i
        t1[m], t2[m], rho[m] = a, b, r
    return t1, t2, rho


def phantom_ellipses_2d(n: int, fov: float, rng: np.random.Generator) -> Phantom:
    """n×n grid, one isochromat per voxel at the voxel centre, z = 0; 4 tissues in nested ellipses."""
    c = grid_coords(n, fov)
    X, Y = np.meshgrid(c, c, indexing="xy")
    lab = _ellipse_labels(_nested_ellipses(rng), X / fov, Y / fov)
    t1, t2, rho = _tissue_params(lab)
    z = np.zeros(X.size)
    return Phantom(X.ravel(), Y.ravel(), z, rho.ravel(), t1.ravel(), t2.ravel(), np.zeros(X.size))


def b0_polynomial_2d(rng: np.random.Generator, fov: float, max_hz: float = 200.0, degree: int = 3):
    """Random 2D polynomial of total degree ≤ 3, scaled to max |Δf| = max_hz on the FOV square."""
    coef = {(i, j): rng.normal() for i in range(degree + 1) for j in range(degree + 1 - i)}
    g = np.linspace(-1, 1, 65)
    U, V = np.meshgrid(g, g)
    ref = sum(c * U**i * V**j for (i, j), c in coef.items())
    scale = max_hz / np.max(np.abs(ref))

    def dw(x, y):
        u, v = 2 * x / fov, 2 * y / fov
        return 2 * math.pi * scale * sum(c * u**i * v**j for (i, j), c in coef.items())

    return dw


def phantom_c2(n: int = 256, iso: int = 4, fov: float = 0.5, rng=None) -> Phantom:
    """2D n×n, `iso` isochromats per voxel with uniform sub-voxel jitter, z = 0.

    Per voxel: half the isochromats are water (tissue T1/T2, Δω0(x)), half are
    fat (T1/T2 = 0.26/0.08 s, Δω0(x) + 2π·FAT_SHIFT_HZ), weighted by a seeded
    fat fraction f ∈ [0, 0.5] so that the voxel's total M0 is the tissue ρ.
    Δω0 is a random polynomial of degree ≤ 3 with max |Δf| = 200 Hz.
    """
    rng = rng_for(2) if rng is None else rng
    if iso % 2:
        raise ValueError("iso must be even (water/fat pairs)")
    ell = _nested_ellipses(rng)
    dw0 = b0_polynomial_2d(rng, fov)
    c = grid_coords(n, fov)
    X, Y = np.meshgrid(c, c, indexing="xy")
    X, Y = X.ravel(), Y.ravel()
    frac = rng.uniform(0.0, 0.5, size=X.size)
    dx = fov / n
    xs = np.repeat(X, iso) + rng.uniform(-0.5, 0.5, size=X.size * iso) * dx
    ys = np.repeat(Y, iso) + rng.uniform(-0.5, 0.5, size=X.size * iso) * dx
    lab = _ellipse_labels(ell, xs / fov, ys / fov)
    t1, t2, rho = _tissue_params(lab)
    is_fat = np.tile(np.arange(iso) >= iso // 2, X.size)
    f = np.repeat(frac, iso)
    w = np.where(is_fat, f, 1.0 - f) / (iso // 2)
    rho = rho * w
    dws = dw0(xs, ys)
    t1 = np.where(is_fat & (lab >= 0), FAT_T1T2[0], t1)
    t2 = np.where(is_fat & (lab >= 0), FAT_T1T2[1], t2)
    dws = np.where(is_fat, dws + 2 * math.pi * FAT_SHIFT_HZ, dws)
    return Phantom(xs, ys, np.zeros_like(xs), rho, t1, t2, dws)


def _blobs(rng, n_blobs=24, fov=0.5, dims=3):
    cen = rng.uniform(-0.3, 0.3, size=(n_blobs, dims)) * fov
    sig = rng.uniform(0.04, 0.12, size=n_blobs) * fov
    amp = rng.uniform(0.3, 1.0, size=n_blobs)
    t1 = rng.uniform(0.2, 2.0, size=n_blobs)
    t2 = np.minimum(rng.uniform(0.02, 0.3, size=n_blobs), t1)
    return cen, sig, amp, t1, t2


def _blob_tissue(pos, blobs, chunk=1 << 20):
    cen, sig, amp, bt1, bt2 = blobs
    n = pos.shape[0]
    rho = np.empty(n)
    t1 = np.empty(n)
    t2 = np.empty(n)
    for s in range(0, n, chunk):
        p = pos[s : s + chunk]
        d2 = ((p[:, None, :] - cen[None, :, :]) ** 2).sum(-1)
        contrib = amp[None, :] * np.exp(-d2 / (2 * sig[None, :] ** 2))
        tot = contrib.sum(1)
        arg = contrib.argmax(1)
        r = np.minimum(tot, 1.0)
        r[r < 0.05] = 0.0
        rho[s : s + chunk] = r
        t1[s : s + chunk] = bt1[arg]
        t2[s : s + chunk] = bt2[arg]
    return rho, t1, t2


def phantom_c3(n: int = 128, iso: int = 2, fov: float = 0.5, rng=None) -> Phantom:
    """3D n³, `iso` isochromats per voxel with sub-voxel jitter; Gaussian-blob tissue map.

    Each blob draws T1 ~ U[0.2, 2] s and T2 ~ U[0.02, 0.3] s (T2 ≤ T1); a spin takes
    the parameters of the blob contributing most at its position, ρ = min(1, Σ blobs)
    (air below 0.05), shared by the voxel's isochromats.  Δω = 0.
    """
    rng = rng_for(3) if rng is None else rng
    blobs = _blobs(rng, fov=fov)
    c = grid_coords(n, fov)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    base = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pos = np.repeat(base, iso, axis=0) + rng.uniform(-0.5, 0.5, size=(base.shape[0] * iso, 3)) * (fov / n)
    rho, t1, t2 = _blob_tissue(pos, blobs)
    return Phantom(pos[:, 0], pos[:, 1], pos[:, 2], rho / iso, t1, t2, np.zeros(pos.shape[0]))


def phantom_random(n_spins: int, fov: float, rng, three_d: bool, density_ref: float) -> Phantom:
    """Uniformly scattered spins (batched workloads): 2D ellipse tissues or 3D blob tissues."""
    if three_d:
        pos = rng.uniform(-0.5, 0.5, size=(n_spins, 3)) * fov
        rho, t1, t2 = _blob_tissue(pos, _blobs(rng, fov=fov))
    else:
        pos = np.zeros((n_spins, 3))
        pos[:, :2] = rng.uniform(-0.5, 0.5, size=(n_spins, 2)) * fov
        lab = _ellipse_labels(_nested_ellipses(rng), pos[:, 0] / fov, pos[:, 1] / fov)
        t1, t2, rho = _tissue_params(lab)
    rho = rho * (density_ref / n_spins)
    return Phantom(pos[:, 0], pos[:, 1], pos[:, 2], rho, t1, t2, np.zeros(n_spins))


# ---------------------------------------------------------------------------
# Sequences
# ---------------------------------------------------------------------------


def sinc_pulse(flip: float, n: int, tbw: float) -> np.ndarray:
    """Hard-pulse approximation of a rect-windowed sinc (Eq. 3.23, §7.2.1): signed sub-pulse flips.

    Sample i sits at u_i = (i + ½)/n − ½ of the pulse; envelope sinc(tbw·u); the
    flips are normalised so that they add up to `flip` (small-tip reading).
    """
    u = (np.arange(n) + 0.5) / n - 0.5
    w = np.sinc(tbw * u)
    return flip * w / w.sum()


def rf_spoil_phases(n: int, inc_deg: float = 117.0) -> np.ndarray:
    """Quadratic RF-spoiling phase φ_k = φ_{k−1} + k·inc (φ_0 = 0), wrapped to [0, 2π)."""
    k = np.arange(n, dtype=np.float64)
    return np.mod(np.deg2rad(inc_deg) * k * (k + 1) / 2.0, 2 * math.pi)


def flash(
    n_read: int,
    n_pe: int,
    fov: float,
    flip: float,
    tr: float,
    te: float,
    dwell: float,
    t_pre: float = 1e-3,
    n_pe2: int = 1,
    gamma: float = GAMMA_BAR,
    rf_spoil: bool = False,
    spoil_cycles: float = 2.0,
    shaped=None,
    tau_rf: float = 10e-6,
    g_slice: float = 0.0,
    name: str = "flash",
) -> Sequence:
    """Gradient-echo (FLASH) Cartesian sequence, 2D (n_pe2 = 1) or 3D.

    Per TR: excitation → prephase/phase-encode event → n_read ADC events at the
    readout gradient → spoiler + phase rewinder until TR.  k-space sample n of a
    line sits at k_x = (n − n_read/2)/fov (cycles/m), line m at k_y = (m − n_pe/2)/fov,
    partition p at k_z = (p − n_pe2/2)/fov.  TE is from the excitation centre to
    the centre sample (n = n_read/2, taken at the end of its ADC event).
    `shaped` (signed sub-pulse flips) replaces the hard pulse by a train of RF
    samples spaced `tau_rf` under `g_slice`.
    """
    dk = 1.0 / fov
    g_read = dk / (gamma * dwell)
    ev = _Events()
    n_tr = n_pe * n_pe2
    phases = rf_spoil_phases(n_tr) if rf_spoil else np.zeros(n_tr)
    to_center = (n_read // 2 + 1) * dwell
    if shaped is None:
        t_wait = te - t_pre - to_center
        exc_len = 0.0
        t_pre_eff = t_pre
    else:
        exc_len = len(shaped) * tau_rf
        t_wait = 0.0
        t_pre_eff = te - exc_len / 2 - to_center
    if t_wait < -1e-12 or t_pre_eff <= 0:
        raise ValueError("TE too short for this readout")
    t_rest = tr - (exc_len + t_wait + t_pre_eff + n_read * dwell)
    if t_rest < -1e-12:
        raise ValueError("TR too short")
    t_rest = max(t_rest, 0.0)
    idx = 0
    for p in range(n_pe2):
        for m in range(n_pe):
            ph = float(phases[idx])
            idx += 1
            if shaped is None:
                ev.add(t_wait, flip=flip, phase=ph)
            else:
                for a in shaped:
                    ev.add(tau_rf, gz=g_slice, flip=float(a), phase=ph)
            kx = -(n_read // 2 + 1) * dk
            ky = (m - n_pe // 2) * dk
            kz = (p - n_pe2 // 2) * dk if n_pe2 > 1 else 0.0
            gz_pre = kz / (gamma * t_pre_eff)
            if shaped is not None:
                # slice refocus: half of the slice-select moment, negative
                gz_pre -= g_slice * exc_len / 2 / t_pre_eff
            ev.add(t_pre_eff, gx=kx / (gamma * t_pre_eff), gy=ky / (gamma * t_pre_eff), gz=gz_pre)
            for _ in range(n_read):
                ev.add(dwell, gx=g_read, adc=1, adc_phase=ph)
            if t_rest > 0:
                k_sp = spoil_cycles * n_read * dk
                ev.add(
                    t_rest,
                    gx=k_sp / (gamma * t_rest),
                    gy=-ky / (gamma * t_rest),
                    gz=-kz / (gamma * t_rest),
                )
    shape = (n_pe2, n_pe, n_read) if n_pe2 > 1 else (n_pe, n_read)
    return Sequence(ev.array(), gamma, shape, name)


def spin_echo(
    n_read: int,
    n_pe: int,
    fov: float,
    te: float,
    tr: float,
    dwell: float,
    n_rf: int = 128,
    tau_rf: float = 20e-6,
    tbw: float = 4.0,
    thk: float = 0.01,
    flip_exc: float = math.pi / 2,
    flip_ref: float = math.pi,
    t_pre: float = 2e-3,
    t_crush: float = 1e-3,
    gamma: float = GAMMA_BAR,
    name: str = "se",
) -> Sequence:
    """2D slice-selective spin echo with sinc excitation (phase 0) and refocusing (phase π/2).

    Per TR: n_rf excitation sub-pulses under the slice gradient → slice refocus +
    phase encode + readout prephase (all before the refocusing pulse, so the
    encodes are negated) → wait → crusher → n_rf refocusing sub-pulses → crusher →
    wait → n_read ADC events → rest.  The refocusing pulse is centred at TE/2, the
    centre sample at TE (times from the excitation centre).
    """
    dk = 1.0 / fov
    g_read = dk / (gamma * dwell)
    half = n_rf * tau_rf / 2
    g_ss = (tbw / (n_rf * tau_rf)) / (gamma * thk)
    g_cr = (2.0 / thk) / (gamma * t_crush)
    a_exc = sinc_pulse(flip_exc, n_rf, tbw)
    a_ref = sinc_pulse(flip_ref, n_rf, tbw)
    wait1 = te / 2 - half - t_crush - (half + t_pre)
    wait2 = te - (n_read // 2 + 1) * dwell - (te / 2 + half + t_crush)
    rest = tr - (te + (n_read // 2 - 1) * dwell + half)
    if min(wait1, wait2) < -1e-12 or rest < -1e-12:
        raise ValueError("TE/TR too short for this spin echo")
    wait1, wait2, rest = max(wait1, 0.0), max(wait2, 0.0), max(rest, 0.0)
    ev = _Events()
    for m in range(n_pe):
        for a in a_exc:
            ev.add(tau_rf, gz=g_ss, flip=float(a), phase=0.0)
        kx = (n_read // 2 + 1) * dk
        ky = -(m - n_pe // 2) * dk
        ev.add(t_pre, gx=kx / (gamma * t_pre), gy=ky / (gamma * t_pre), gz=-g_ss * half / t_pre)
        ev.add(wait1)
        ev.add(t_crush, gz=g_cr)
        for a in a_ref:
            ev.add(tau_rf, gz=g_ss, flip=float(a), phase=math.pi / 2)
        ev.add(t_crush, gz=g_cr)
        ev.add(wait2)
        for _ in range(n_read):
            ev.add(dwell, gx=g_read, adc=1)
        ev.add(rest)
    return Sequence(ev.array(), gamma, (n_pe, n_read), name)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------


def config1(seed=None) -> Workload:
    """2D 64² FLASH, 1 iso/voxel (4096 spins), 15°, TR 10 ms, TE 5 ms, dwell 10 µs."""
    rng = rng_for(1, seed)
    ph = phantom_ellipses_2d(64, 0.5, rng)
    seq = flash(64, 64, 0.5, math.radians(15), 10e-3, 5e-3, 10e-6, name="flash2d-64")
    return Workload("c1_flash2d_64", ph, seq, "4 tissues in seeded nested ellipses, Δω = 0")


def config2(seed=None, n: int = 256, iso: int = 4) -> Workload:
    """2D 256² spin echo, 4 iso/voxel, sinc 90/180 (TBW 4, 128 samples), B0 + fat."""
    rng = rng_for(2, seed)
    ph = phantom_c2(n, iso, 0.5, rng)
    seq = spin_echo(n, n, 0.5, 50e-3, 500e-3, 40e-6, name=f"se2d-{n}")
    return Workload(f"c2_se2d_{n}", ph, seq, "jittered isochromats, fat fraction, B0 polynomial ±200 Hz")


def config2_legendre(seed=None, n: int = 256, iso: int = 4, c_tesla: float = 20e-6, radius: float = 0.25) -> Workload:
    """C2 with the static-field inhomogeneity of a whole-body magnet (Eq. 6.3) in place of the
    random polynomial: C = 20 µT and a homogeneity sphere of diameter 0.5 m (the values of §7.1.2
    and Fig. 6.2); fat isochromats keep their chemical shift."""
    w = config2(seed, n, iso)
    ph = w.phantom
    fat = np.zeros(ph.n, dtype=bool)
    fat[np.tile(np.arange(iso) >= iso // 2, ph.n // iso)] = True
    dw = dw_from_b0(b0_legendre(ph.x, ph.y, ph.z, c_tesla, radius)) + np.where(fat, 2 * math.pi * FAT_SHIFT_HZ, 0.0)
    return Workload(f"c2_se2d_{n}_legendre", Phantom(ph.x, ph.y, ph.z, ph.rho, ph.t1, ph.t2, dw), w.sequence,
                    f"Eq. 6.3 inhomogeneity C = {c_tesla * 1e6:g} uT, R = {radius:g} m, plus fat shift")


def concomitant_transverse(events) -> np.ndarray:
    """Transverse components of the gradient field that Maxwell's equations require beside an
    ideal z-field (G.x) e_z (§3.4.3.2 names them concomitant gradients): the curl- and
    divergence-free completion B = (-Gz x/2 + Gx z, -Gz y/2 + Gy z, G.x), i.e. per event
    gtx = (-Gz/2, 0, Gx) and gty = (0, -Gz/2, Gy) [T/m], as [n_events, 6]."""
    ev = events
    gt = np.zeros((len(ev), 6))
    gt[:, 0] = -0.5 * ev["gz"]
    gt[:, 2] = ev["gx"]
    gt[:, 4] = -0.5 * ev["gz"]
    gt[:, 5] = ev["gy"]
    return gt


def tilted_field_directions(ph: Phantom, max_tilt: float, rng: np.random.Generator) -> np.ndarray:
    """Unit static-field directions per spin (§3.2): a seeded smooth tilt, polar angle linear in
    position up to max_tilt at the edge of a 0.5 m field of view, azimuth a seeded linear field;
    [n_spins, 3]."""
    c = rng.uniform(-1, 1, 6)
    tilt = max_tilt * np.clip(np.abs(c[0] * ph.x + c[1] * ph.y + c[2] * ph.z) / (0.25 * np.abs(c[:3]).sum()), 0, 1)
    az = math.pi * (c[3] * ph.x + c[4] * ph.y + c[5] * ph.z) / 0.25
    return np.stack([np.sin(tilt) * np.cos(az), np.sin(tilt) * np.sin(az), np.cos(tilt)], axis=1)


@dataclasses.dataclass
class FieldWorkload:
    name: str
    phantom: Phantom
    sequence: Sequence
    b0_dir: np.ndarray       # [n_spins, 3]
    g_transverse: np.ndarray  # [n_events, 6]
    b0_tesla: float

    @property
    def spin_steps(self) -> int:
        return self.phantom.n * self.sequence.n_events


def config_fields(seed=None, base: str = "c1", b0_tesla: float | None = None,
                  max_tilt: float = math.radians(10.0)) -> FieldWorkload:
    """Non-parallel fields: a static field whose direction tilts smoothly by up to 10° across the
    object, and the Maxwell concomitant components of every gradient, on
      base "c1": the 64² FLASH at a low main field (0.05 T, where concomitant fields matter), or
      base "c2": the 256² spin echo with B0 polynomial and fat at 1.5 T (the field its fat shift
                 belongs to)."""
    w = {"c1": config1, "c2": config2}[base](seed)
    b0 = b0_tesla if b0_tesla is not None else {"c1": 0.05, "c2": 1.5}[base]
    rng = rng_for(7, seed)
    nd = tilted_field_directions(w.phantom, max_tilt, rng)
    stem = {"c1": "flash2d_64", "c2": "se2d_256"}[base]
    return FieldWorkload(f"fields_{stem}_b0_{b0:g}T", w.phantom, w.sequence, nd,
                         concomitant_transverse(w.sequence.events), b0)


def config3(seed=None, n: int = 128, iso: int = 2) -> Workload:
    """3D n³ RF-spoiled GRE, 2 iso/voxel, 10°, TR 8 ms, TE 4 ms, dwell 10 µs."""
    rng = rng_for(3, seed)
    ph = phantom_c3(n, iso, 0.5, rng)
    seq = flash(n, n, 0.5, math.radians(10), 8e-3, 4e-3, 10e-6, n_pe2=n, rf_spoil=True, name=f"spgr3d-{n}")
    return Workload(f"c3_spgr3d_{n}", ph, seq, "Gaussian-blob tissue map, Δω = 0")


def config4(seed=None, n_phantoms: int = 64, min_spins: float = 1e4, max_spins: float = 2e6):
    """64 independent phantoms (log-uniform spin counts) with their own FLASH or SE sequences."""
    rng = rng_for(4, seed)
    out = []
    for i in range(n_phantoms):
        n_spins = int(round(math.exp(rng.uniform(math.log(min_spins), math.log(max_spins)))))
        three_d = n_spins > 256 * 256 * 4
        N = int(rng.choice([64, 128, 256]))
        flip = math.radians(rng.uniform(5.0, 90.0))
        tr = math.exp(rng.uniform(math.log(5e-3), math.log(500e-3)))
        ph = phantom_random(n_spins, 0.5, rng, three_d, density_ref=float(N * N))
        if rng.uniform() < 0.5:
            dwell = 10e-6
            te = max(1e-3 + (N // 2 + 1) * dwell, round(tr / 2 / 1e-5) * 1e-5)
            te = min(te, 10e-3 + (N // 2 + 1) * dwell)
            tr_eff = max(tr, te + N * dwell)
            seq = flash(N, N, 0.5, flip, tr_eff, te, dwell, name=f"flash2d-{N}")
        else:
            dwell = 10e-6
            half, t_pre, t_cr = 128 * 20e-6 / 2, 2e-3, 1e-3
            te = 2 * max(2 * half + t_cr + t_pre, (N // 2 + 1) * dwell + half + t_cr)
            te = math.ceil(te / 1e-5) * 1e-5
            tr_eff = max(tr, te + (N // 2) * dwell + half + 1e-4)
            seq = spin_echo(N, N, 0.5, te, tr_eff, dwell, flip_exc=flip, name=f"se2d-{N}")
        out.append(Workload(f"c4_{i:02d}", ph, seq, f"{'3D' if three_d else '2D'} {n_spins} spins"))
    return out


def config5(seed=None, n: int = 128, n_rf: int = 256):
    """2D 128² FLASH with a learnable 256-sample RF waveform (10 µs per sample).

    Returns (workload with the initial waveform, target phantom, initial RF flips).
    The target phantom is the same geometry with per-spin ρ ±5 %, T1/T2 ±10 %.
    """
    rng = rng_for(5, seed)
    ph = phantom_ellipses_2d(n, 0.5, rng)
    rf = sinc_pulse(math.radians(15), n_rf, 4.0)
    g_ss = (4.0 / (n_rf * 10e-6)) / (GAMMA_BAR * 0.01)
    seq = flash(n, n, 0.5, 0.0, 10e-3, 5e-3, 10e-6, shaped=rf, tau_rf=10e-6, g_slice=g_ss, name=f"flash2d-rf-{n}")
    tgt = Phantom(
        ph.x,
        ph.y,
        ph.z,
        ph.rho * rng.uniform(0.95, 1.05, ph.n),
        ph.t1 * rng.uniform(0.9, 1.1, ph.n),
        ph.t2 * rng.uniform(0.9, 1.1, ph.n),
        ph.dw,
    )
    return Workload(f"c5_flash2d_rf_{n}", ph, seq, "learnable RF amplitudes"), tgt, rf


def rf_event_index(seq: Sequence) -> np.ndarray:
    """Indices of the events that carry an RF sub-pulse (α ≠ 0)."""
    return np.nonzero(seq.events["rf_flip"] != 0.0)[0]


def with_rf_waveform(seq: Sequence, waveform: np.ndarray) -> Sequence:
    """Copy of a shaped-excitation sequence whose RF samples (per TR) are replaced by `waveform`."""
    ev = seq.events.copy()
    idx = rf_event_index(seq)
    n_rf = len(waveform)
    if idx.size % n_rf:
        raise ValueError("RF event count is not a multiple of the waveform length")
    ev["rf_flip"][idx] = np.tile(np.asarray(waveform, dtype=np.float64), idx.size // n_rf)
    return Sequence(ev, seq.gamma_hz_per_t, seq.kshape, seq.name)


def rasterize(seq: Sequence, raster: float = 10e-6) -> Sequence:
    """Stress variant of a sequence: every event longer than `raster` becomes ceil(Δt/raster)
    consecutive events of equal length with the same gradient; the RF pulse stays on the first
    piece (it acts at the start of the event) and the ADC sample on the last (it is taken at the
    end).  Precession angles and relaxation over the pieces compose to those of the whole event
    (Eq. 4.1 applied piecewise), so the signal is unchanged; only the number of events grows
    (the 10 µs piecewise-constant reading of the event lists)."""
    ev = seq.events
    n = np.maximum(1, np.ceil(ev["dt"] / raster * (1.0 - 1e-9))).astype(np.int64)
    out = np.repeat(ev, n)
    out["dt"] = np.repeat(ev["dt"] / n, n)
    start = np.concatenate([[0], np.cumsum(n)[:-1]])
    not_first = np.ones(out.shape[0], dtype=bool)
    not_first[start] = False
    not_last = np.ones(out.shape[0], dtype=bool)
    not_last[start + n - 1] = False
    out["rf_flip"][not_first] = 0.0
    out["rf_phase"][not_first] = 0.0
    out["adc"][not_last] = 0
    out["adc_phase"][not_last] = 0.0
    return Sequence(out, seq.gamma_hz_per_t, seq.kshape, (seq.name or "seq") + f"_rasterized{raster * 1e6:g}us")


# ---------------------------------------------------------------------------
# Small random cases (parity tests, edge cases)
# ---------------------------------------------------------------------------


def random_phantom(n: int, rng: np.random.Generator, fov: float = 0.5, inf_frac: float = 0.1) -> Phantom:
    x = rng.uniform(-fov / 2, fov / 2, n)
    y = rng.uniform(-fov / 2, fov / 2, n)
    z = rng.uniform(-fov / 8, fov / 8, n)
    rho = rng.uniform(0.0, 1.0, n)
    t1 = rng.uniform(0.05, 3.0, n)
    t2 = np.minimum(rng.uniform(0.01, 0.5, n), t1)
    t1[rng.uniform(size=n) < inf_frac] = np.inf
    t2[rng.uniform(size=n) < inf_frac] = np.inf
    dw = 2 * math.pi * rng.uniform(-300.0, 300.0, n)
    return Phantom(x, y, z, rho, t1, t2, dw)


def random_sequence(n_events: int, rng: np.random.Generator, fov: float = 0.5, runs: bool = True) -> Sequence:
    """Random event list exercising every event feature.

    Mixes hard pulses of any flip/phase, zero-length events, free precession
    with random gradients, isolated ADC events with random demodulation phases
    and (with `runs`) constant-gradient ADC runs and repeated RF sub-pulse trains,
    the structures real sequences are made of.
    """
    ev = _Events()
    dk = 1.0 / fov
    while len(ev.rows) < n_events:
        kind = rng.integers(0, 6 if runs else 3)
        if kind == 0:  # hard pulse, maybe zero length
            dt = 0.0 if rng.uniform() < 0.3 else rng.uniform(1e-5, 5e-3)
            ev.add(dt, *(rng.normal(size=3) * 5e-3), flip=rng.uniform(-math.pi, math.pi), phase=rng.uniform(0, 2 * math.pi))
        elif kind == 1:  # free precession
            ev.add(rng.uniform(0, 10e-3), *(rng.normal(size=3) * 5e-3))
        elif kind == 2:  # isolated ADC
            ev.add(rng.uniform(1e-6, 1e-4), *(rng.normal(size=3) * 5e-3), adc=1, adc_phase=rng.uniform(0, 2 * math.pi))
        elif kind == 3:  # ADC run
            n = int(rng.integers(1, 70))
            g = dk / (GAMMA_BAR * 10e-6) * rng.uniform(-1, 1)
            ph = rng.uniform(0, 2 * math.pi)
            for _ in range(n):
                ev.add(10e-6, gx=g, adc=1, adc_phase=ph)
        elif kind == 4:  # RF sub-pulse train
            n = int(rng.integers(2, 40))
            gz = rng.uniform(0, 5e-3)
            ph = rng.uniform(0, 2 * math.pi)
            for a in sinc_pulse(rng.uniform(0, math.pi), n, 4.0):
                ev.add(20e-6, gz=gz, flip=float(a), phase=ph)
        else:  # repeated identical free-precession intervals
            n = int(rng.integers(2, 6))
            dt = rng.uniform(0, 3e-3)
            g = rng.normal(size=3) * 3e-3
            for _ in range(n):
                ev.add(dt, *g)
    return Sequence(ev.array()[:n_events], GAMMA_BAR, (), "random")


# ---------------------------------------------------------------------------
# K-t formalism inputs (§4.2): ensembles (a dictionary over T1, T2, B1, Δf) and step lists
# ---------------------------------------------------------------------------

KT_STEP_DTYPE = np.dtype([("alpha", "<f8"), ("phi", "<f8"), ("tau", "<f8"), ("adc_phase", "<f8"),
                          ("shift", "<i4"), ("sample", "<i4")])
assert KT_STEP_DTYPE.itemsize == 40


def kt_steps(rows) -> np.ndarray:
    """Rows of (alpha, phi, tau, shift, sample, adc_phase) → KT_STEP_DTYPE array."""
    out = np.zeros(len(rows), dtype=KT_STEP_DTYPE)
    for k, (al, ph, tau, q, smp, adc) in enumerate(rows):
        out[k] = (al, ph, tau, adc, q, smp)
    return out


@dataclasses.dataclass
class KtDictionary:
    t1: np.ndarray
    t2: np.ndarray
    b1: np.ndarray
    df: np.ndarray

    @property
    def n(self) -> int:
        return int(self.t1.shape[0])


def kt_dictionary(n: int, rng: np.random.Generator, off_resonance: bool = True) -> KtDictionary:
    """Seeded ensemble parameters: T1 log-U[0.1, 4] s, T2 log-U[0.01, 1] s (<= T1), B1 U[0.7, 1.3],
    Δf U[-50, 50] Hz (0 without off-resonance)."""
    t1 = np.exp(rng.uniform(math.log(0.1), math.log(4.0), n))
    t2 = np.minimum(np.exp(rng.uniform(math.log(0.01), math.log(1.0), n)), t1)
    b1 = rng.uniform(0.7, 1.3, n)
    df = rng.uniform(-50.0, 50.0, n) if off_resonance else np.zeros(n)
    return KtDictionary(t1, t2, b1, df)


def kt_fingerprint_sequence(n_tr: int, rng: np.random.Generator) -> np.ndarray:
    """Fingerprinting-style train: an inversion, then n_tr pulses with a smoothly varying flip
    (5°..70°), alternating phase, TR U[10, 15] ms, one order of unbalanced gradient per TR and a
    sample every TR (receiver phase = pulse phase)."""
    rows = [(math.pi, 0.0, 20e-3, 0, 0, 0.0)]
    for k in range(n_tr):
        al = math.radians(5.0 + 65.0 * abs(math.sin(math.pi * k / 250.0)))
        ph = math.pi * (k % 2)
        rows.append((al, ph, rng.uniform(10e-3, 15e-3), 1, 1, ph))
    return kt_steps(rows)


def kt_random_sequence(n_steps: int, rng: np.random.Generator, max_shift: int = 2) -> np.ndarray:
    """Random flips and phases, intervals, order shifts in [-max_shift, max_shift], random samples."""
    rows = []
    for _ in range(n_steps):
        al = rng.uniform(-math.pi, math.pi) if rng.uniform() < 0.8 else 0.0
        rows.append((al, rng.uniform(0, 2 * math.pi), rng.uniform(0.0, 8e-3), int(rng.integers(-max_shift, max_shift + 1)),
                     int(rng.uniform() < 0.6), rng.uniform(0, 2 * math.pi)))
    return kt_steps(rows)


# ---------------------------------------------------------------------------
# Static-field inhomogeneity of a whole-body magnet (Eq. 6.3)
# ---------------------------------------------------------------------------


def legendre(n: int, x):
    """Legendre polynomial P_n(x) by the three-term (Bonnet) recursion."""
    x = np.asarray(x, dtype=float)
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    return p1


def b0_legendre(x, y, z, c_tesla: float, radius: float) -> np.ndarray:
    """ΔB0 [T] of Eq. 6.3: -C·(r/R)^12·P12(cos θ), r = |x|, θ the declination from the z axis."""
    x, y, z = (np.asarray(a, dtype=float) for a in (x, y, z))
    r = np.sqrt(x * x + y * y + z * z)
    cos_t = np.divide(z, r, out=np.ones_like(r), where=r > 0)
    return -c_tesla * (r / radius) ** 12 * legendre(12, cos_t)


def dw_from_b0(delta_b0, gamma_hz_per_t: float = GAMMA_BAR) -> np.ndarray:
    """Off-resonance [rad/s] of a field deviation along z: Δω0 = +γ·ΔB0.

    The simulation turns a spin by θ = (γ G·x + Δω)·Δt, Mxy <- Mxy·exp(-jθ): Δω enters exactly as
    a gradient's field G·x does, i.e. Δω/γ is a field along z in the same sense as G·x (the Bloch
    equation in the rotating frame, Eqs. 3.11, 3.13).  So a deviation ΔB0 of the static field
    enters as +γ·ΔB0, and a spin at the centre in a deviation equal to G·x0 precesses like a spin
    at x0 in the gradient G.  (Eq. 6.1 writes ω = -γB with the opposite orientation of the
    angle; the library's Δω is the clockwise-positive frequency of its precession matrices.)"""
    return 2 * math.pi * gamma_hz_per_t * np.asarray(delta_b0, dtype=float)
