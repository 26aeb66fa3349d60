"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each ``pin_*`` takes a simulator with the oracle's calling convention
``sim(phantom, events, gamma, m_init=None, want_signal=True, want_state=False)``
and raises AssertionError if the simulator disagrees with an independent
statement of the physics:

* the Bloch ODE itself (Eqs. A.1-A.4, A.12) integrated exactly by a matrix
  exponential for piecewise-constant fields (scipy.linalg.expm),
* the rotation sense of the hard pulse via scipy's Rodrigues rotation,
* closed forms: FID, T1 recovery / inversion null, the spin echo,
* the paper's worked example Eq. 4.6 (tests/golden/worked_example_4_6.txt),
* the imaging equation Eq. 3.33 against numpy's FFT,
* the K-t / extended-phase-graph recursion of §4.2.2 (Eqs. 4.2, 4.14-4.17),
* invariants: linearity in ρ, additivity over spin subsets, permutation.

The pins are chosen so that a plausible mistake in the oracle (a flipped sign,
a transposed matrix, a dropped term, a wrong index) fails at least one of them;
``test_oracle_mutations.py`` plants such mistakes and checks exactly that.
"""
from __future__ import annotations

import math
import os

import numpy as np
from scipy.linalg import expm
from scipy.spatial.transform import Rotation

from paper_1305_6861_gb300.workloads import GAMMA_BAR, Phantom, make_events

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _ph(x, y=None, z=None, rho=None, t1=None, t2=None, dw=None):
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = x.shape[0]
    f = lambda v, d: np.full(n, d) if v is None else np.broadcast_to(np.asarray(v, dtype=float), (n,)).copy()
    return Phantom(x, f(y, 0.0), f(z, 0.0), f(rho, 1.0), f(t1, np.inf), f(t2, np.inf), f(dw, 0.0))


# --- brute force: the Bloch ODE with piecewise-constant fields ------------------------------


def _free_generator(gamma, bz, t1, t2, m0):
    """Augmented 4×4 generator of dM/dt = A M + f for a static field along z (Eqs. A.2-A.4)."""
    r1 = 0.0 if math.isinf(t1) else 1.0 / t1
    r2 = 0.0 if math.isinf(t2) else 1.0 / t2
    A = np.zeros((4, 4))
    A[0, 0] = -r2
    A[0, 1] = gamma * bz
    A[1, 0] = -gamma * bz
    A[1, 1] = -r2
    A[2, 2] = -r1
    A[2, 3] = m0 * r1
    return A


def _rf_generator(phi):
    """Rotating-frame B1 generator of Eq. A.12 per unit flip (on resonance, relaxation neglected)."""
    s, c = math.sin(phi), math.cos(phi)
    K = np.zeros((4, 4))
    K[0, 2] = -s
    K[1, 2] = c
    K[2, 0] = s
    K[2, 1] = -c
    return K


def bloch_bruteforce(ph: Phantom, events, gamma_hz, m_init=None):
    """Exact solution of the Bloch ODE for a piecewise-constant event list, spin by spin."""
    gamma = 2 * math.pi * gamma_hz
    n = ph.n
    n_adc = int(np.count_nonzero(events["adc"]))
    sig = np.zeros(n_adc, dtype=complex)
    final = np.zeros((n, 3))
    for s in range(n):
        v = np.array([0.0, 0.0, ph.rho[s], 1.0])
        if m_init is not None:
            v[:3] = m_init[s]
        j = 0
        for e in events:
            if e["rf_flip"] != 0.0:
                v = expm(e["rf_flip"] * _rf_generator(e["rf_phase"])) @ v
            # local field along z in the rotating frame: G·x + Δω/γ  (Eqs. 3.11, 3.13)
            bz = e["gx"] * ph.x[s] + e["gy"] * ph.y[s] + e["gz"] * ph.z[s] + ph.dw[s] / gamma
            v = expm(e["dt"] * _free_generator(gamma, bz, ph.t1[s], ph.t2[s], ph.rho[s])) @ v
            if e["adc"]:
                sig[j] += (v[0] + 1j * v[1]) * np.exp(-1j * e["adc_phase"])
                j += 1
        final[s] = v[:3]
    return sig, final


def _close(a, b, tol, what):
    a = np.asarray(a)
    b = np.asarray(b)
    err = np.max(np.abs(a - b)) if a.size else 0.0
    scale = max(1.0, float(np.max(np.abs(b))) if b.size else 1.0)
    assert err <= tol * scale, f"{what}: max |diff| = {err:.3e} (tol {tol * scale:.1e})"


# --- pins ------------------------------------------------------------------------------------


def pin_rf_rotation(sim):
    """Eq. 3.19 = rotation by −α about (cos φ, sin φ, 0) = exp of the Eq. A.12 generator."""
    rng = np.random.default_rng(11)
    for _ in range(12):
        a, phi = rng.uniform(-math.pi, math.pi), rng.uniform(0, 2 * math.pi)
        m0 = rng.normal(size=(4, 3))
        ph = _ph(np.zeros(4))
        ev = make_events([(0.0, 0, 0, 0, a, phi, 0, 0.0)])
        _, out = sim(ph, ev, GAMMA_BAR, m_init=m0, want_signal=False, want_state=True)
        ref = Rotation.from_rotvec(-a * np.array([math.cos(phi), math.sin(phi), 0.0])).apply(m0)
        _close(out, ref, 1e-13, "hard pulse vs Rodrigues rotation")
        ref2 = (expm(a * _rf_generator(phi))[:3, :3] @ m0.T).T
        _close(out, ref2, 1e-13, "hard pulse vs exp(A.12)")


def pin_special_flips(sim):
    """90°x: (0,0,M0) → (0,M0,0); 180°: Mz → −M0; 180°x conjugates Mxy (Eq. 4.2 with α = π)."""
    ph = _ph([0.0], rho=[0.7])
    _, m = sim(ph, make_events([(0.0, 0, 0, 0, math.pi / 2, 0.0, 0, 0.0)]), GAMMA_BAR, want_signal=False, want_state=True)
    _close(m[0], [0.0, 0.7, 0.0], 1e-15, "90°x")
    _, m = sim(ph, make_events([(0.0, 0, 0, 0, math.pi, 1.3, 0, 0.0)]), GAMMA_BAR, want_signal=False, want_state=True)
    _close(m[0], [0.0, 0.0, -0.7], 1e-15, "180°")
    m0 = np.array([[0.3, -0.4, 0.2]])
    _, m = sim(ph, make_events([(0.0, 0, 0, 0, math.pi, 0.0, 0, 0.0)]), GAMMA_BAR, m_init=m0, want_signal=False, want_state=True)
    _close(m[0], [0.3, 0.4, -0.2], 1e-15, "180°x conjugation")
    # phase 90°: the tipped magnetisation points along −x (M_x = −M0 sin α)
    _, m = sim(ph, make_events([(0.0, 0, 0, 0, 0.4, math.pi / 2, 0, 0.0)]), GAMMA_BAR, want_signal=False, want_state=True)
    _close(m[0], [-0.7 * math.sin(0.4), 0.0, 0.7 * math.cos(0.4)], 1e-15, "phase 90°")


def pin_free_precession_expm(sim):
    """Free precession + relaxation over Δt = exact ODE solution (Eqs. 3.5/3.14 vs A.2-A.4)."""
    rng = np.random.default_rng(12)
    n = 6
    ph = Phantom(rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, n), rng.uniform(-0.05, 0.05, n),
                 rng.uniform(0.1, 1.0, n), rng.uniform(0.1, 2.0, n), rng.uniform(0.01, 0.2, n),
                 2 * math.pi * rng.uniform(-200, 200, n))
    ph.t1[0] = np.inf
    ph.t2[1] = np.inf
    rows = [(rng.uniform(1e-4, 5e-3), *(rng.normal(size=3) * 4e-3), 0.0, 0.0, 1, rng.uniform(0, 6.3)) for _ in range(5)]
    ev = make_events(rows)
    m0 = rng.normal(size=(n, 3))
    sig, st = sim(ph, ev, GAMMA_BAR, m_init=m0, want_state=True)
    rs, rst = bloch_bruteforce(ph, ev, GAMMA_BAR, m_init=m0)
    _close(st, rst, 1e-11, "free precession state vs expm")
    _close(sig, rs, 1e-11, "free precession signal vs expm")


def pin_bruteforce_sequences(sim):
    """Random sequences (pulses, gradients, Δt = 0, T = ∞, ADC phases) vs the exact ODE solution."""
    from paper_1305_6861_gb300.workloads import random_phantom, random_sequence

    rng = np.random.default_rng(13)
    for trial in range(3):
        ph = random_phantom(4, rng)
        seq = random_sequence(40, rng, runs=(trial > 0))
        sig, st = sim(ph, seq.events, seq.gamma_hz_per_t, want_state=True)
        rs, rst = bloch_bruteforce(ph, seq.events, seq.gamma_hz_per_t)
        _close(st, rst, 1e-10, "random sequence final state vs expm")
        _close(sig, rs, 1e-10, "random sequence signal vs expm")


def pin_fid(sim):
    """FID after a 90°x pulse: s(t) = j Σ M0 e^{−t/T2} e^{−jΔω t}, t = (j+1)·Δt (sample at the step's end)."""
    rng = np.random.default_rng(14)
    n = 5
    ph = _ph(rng.uniform(-0.2, 0.2, n), rho=rng.uniform(0.2, 1, n), t1=rng.uniform(0.3, 2, n),
             t2=rng.uniform(0.02, 0.2, n), dw=2 * math.pi * rng.uniform(-100, 100, n))
    dt, ns = 1e-3, 30
    ev = make_events([(0.0, 0, 0, 0, math.pi / 2, 0.0, 0, 0.0)] + [(dt, 0, 0, 0, 0, 0, 1, 0.0)] * ns)
    sig, _ = sim(ph, ev, GAMMA_BAR)
    t = (np.arange(ns) + 1) * dt
    ref = (1j * ph.rho[None, :] * np.exp(-t[:, None] / ph.t2[None, :]) * np.exp(-1j * ph.dw[None, :] * t[:, None])).sum(1)
    _close(sig, ref, 1e-13, "FID closed form")


def pin_t1_recovery(sim):
    """Inversion recovery M_z(TI) = M0(1 − 2e^{−TI/T1}), null at TI = T1 ln 2; saturation recovery."""
    t1s = np.array([0.3, 0.8, 1.2, 4.0])
    ph = _ph(np.zeros(4), rho=[0.7, 0.8, 0.9, 1.0], t1=t1s, t2=[0.04, 0.08, 0.1, 2.0])
    for ti in (0.05, 0.3, 1.0):
        ev = make_events([(ti, 0, 0, 0, math.pi, 0.0, 0, 0.0), (0.0, 0, 0, 0, math.pi / 2, 0.0, 1, 0.0)])
        sig, _ = sim(ph, ev, GAMMA_BAR)
        _close(sig, [1j * np.sum(ph.rho * (1 - 2 * np.exp(-ti / t1s)))], 1e-14, "inversion recovery")
    for k in range(4):
        one = _ph([0.0], rho=[1.0], t1=[t1s[k]], t2=[0.05])
        ev = make_events([(t1s[k] * math.log(2), 0, 0, 0, math.pi, 0.0, 0, 0.0), (0.0, 0, 0, 0, math.pi / 2, 0.0, 1, 0.0)])
        sig, _ = sim(one, ev, GAMMA_BAR)
        assert abs(sig[0]) < 1e-14, f"inversion null at T1 ln 2 missed: {sig[0]}"
    ev = make_events([(0.37, 0, 0, 0, math.pi / 2, 0.0, 0, 0.0)])
    _, st = sim(ph, ev, GAMMA_BAR, want_signal=False, want_state=True)
    _close(st[:, 2], ph.rho * (1 - np.exp(-0.37 / t1s)), 1e-14, "saturation recovery")


def pin_spin_echo(sim):
    """90°x – τ – 180°x – τ: Mxy = −j M0 e^{−2τ/T2} for every Δω and gradient (Fig. 4.7)."""
    rng = np.random.default_rng(15)
    n = 16
    ph = _ph(rng.uniform(-0.2, 0.2, n), y=rng.uniform(-0.2, 0.2, n), rho=rng.uniform(0.2, 1, n),
             t1=rng.uniform(0.3, 2, n), t2=rng.uniform(0.02, 0.2, n), dw=2 * math.pi * rng.uniform(-300, 300, n))
    tau = 7e-3
    g = (3e-3, -2e-3, 0.0)
    ev = make_events([(tau, *g, math.pi / 2, 0.0, 0, 0.0), (tau, *g, math.pi, 0.0, 1, 0.0)])
    sig, st = sim(ph, ev, GAMMA_BAR, want_state=True)
    _close(st[:, 0] + 1j * st[:, 1], -1j * ph.rho * np.exp(-2 * tau / ph.t2), 1e-12, "spin echo per spin")
    _close(sig, [np.sum(-1j * ph.rho * np.exp(-2 * tau / ph.t2))], 1e-12, "spin echo signal")


def load_worked_example():
    rows = []
    with open(os.path.join(GOLDEN, "worked_example_4_6.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            comp, order, expr = line.split(None, 2)
            rows.append((comp, int(order), expr))
    return rows


def pin_worked_example_4_6(sim):
    """Eq. 4.6: two pulses with one gradient moment Δk_x per interval, relaxation neglected."""
    rows = load_worked_example()
    dk, dt = 7.0, 2e-3  # cycles/m, s
    gx = dk / (GAMMA_BAR * dt)
    x = np.linspace(-0.2, 0.2, 9)
    ph = _ph(x)
    for a1, a2 in ((0.3, 1.1), (math.pi / 2, math.pi), (2.0, -0.7)):
        ev = make_events([(dt, gx, 0, 0, a1, 0.0, 0, 0.0), (dt, gx, 0, 0, a2, 0.0, 0, 0.0)])
        _, st = sim(ph, ev, GAMMA_BAR, want_signal=False, want_state=True)
        env = {"sin": np.sin, "cos": np.cos, "a1": a1, "a2": a2}
        ref = {"Mxy": 0j, "Mxyc": 0j, "Mz": 0j}
        for comp, q, expr in rows:
            ref[comp] = ref[comp] + eval(expr, {"__builtins__": {}}, env) * np.exp(-2j * math.pi * q * dk * x)
        mxy = st[:, 0] + 1j * st[:, 1]
        _close(mxy, ref["Mxy"], 1e-13, "Eq. 4.6 Mxy")
        _close(np.conj(mxy), ref["Mxyc"], 1e-13, "Eq. 4.6 Mxy*")
        _close(st[:, 2], ref["Mz"], 1e-13, "Eq. 4.6 Mz")


def pin_imaging_equation(sim):
    """One 90° excitation, T = ∞, Δω = 0, grid spins: s(k) = j Σ ρ e^{−2πj k·x} (Eq. 3.33) = FFT."""
    rng = np.random.default_rng(16)
    N, fov = 16, 0.5
    c = (np.arange(N) - N // 2) * fov / N
    X, Y = np.meshgrid(c, c, indexing="xy")
    rho = rng.uniform(0, 1, (N, N))
    ph = _ph(X.ravel(), y=Y.ravel(), rho=rho.ravel())
    dk = 1.0 / fov
    dwell, tm = 10e-6, 1e-3
    gr = dk / (GAMMA_BAR * dwell)
    rows = [(0.0, 0, 0, 0, math.pi / 2, 0.0, 0, 0.0)]
    kx, ky = 0.0, 0.0
    for m in range(N):
        tx, ty = -(N // 2 + 1) * dk, (m - N // 2) * dk
        rows.append((tm, (tx - kx) / (GAMMA_BAR * tm), (ty - ky) / (GAMMA_BAR * tm), 0, 0, 0, 0, 0.0))
        rows += [(dwell, gr, 0, 0, 0, 0, 1, 0.0)] * N
        kx, ky = tx + N * dk, ty
    sig, _ = sim(ph, make_events(rows), GAMMA_BAR)
    ref = 1j * np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(rho)))
    _close(sig.reshape(N, N), ref, 1e-11, "imaging equation vs FFT")


def epg_signal(alphas, phis, tau, t1, t2, orders):
    """K-t formalism (§4.2.2): configuration populations under Eq. 4.2 (RF), Eq. 4.17 (one
    order shift per interval) and Eqs. 4.15/4.16 (relaxation); returns F_0 after each interval."""
    K = orders
    F = np.zeros(2 * K + 1, dtype=complex)
    Z = np.zeros(2 * K + 1, dtype=complex)
    Z[K] = 1.0
    e1, e2 = math.exp(-tau / t1), math.exp(-tau / t2)
    out = []
    for a, p in zip(alphas, phis):
        c2, s2 = math.cos(a / 2) ** 2, math.sin(a / 2) ** 2
        sa = math.sin(a)
        T = np.array([
            [c2, s2 * np.exp(2j * p), sa * np.exp(1j * (p + math.pi / 2))],
            [s2 * np.exp(-2j * p), c2, sa * np.exp(-1j * (p + math.pi / 2))],
            [sa / 2 * np.exp(-1j * (p - math.pi / 2)), sa / 2 * np.exp(1j * (p - math.pi / 2)), math.cos(a)],
        ])
        Fc = np.conj(F[::-1])  # population of Mxy* at order i is conj(F_{-i})
        F, Z = T[0, 0] * F + T[0, 1] * Fc + T[0, 2] * Z, T[2, 0] * F + T[2, 1] * Fc + T[2, 2] * Z
        assert abs(F[-1]) == 0.0, "configuration order overflow"
        F = np.roll(F, 1)
        F *= e2
        Z *= e1
        Z[K] += 1.0 - e1
        out.append(F[K])
    return np.array(out)


def pin_epg_cross_check(sim):
    """N isochromats spread over one gradient cycle: Σ_s Mxy/N = F_0 of the K-t recursion while
    every populated order stays below N (discrete orthogonality)."""
    rng = np.random.default_rng(17)
    N, P = 64, 14
    dk, tau = 5.0, 4e-3
    x = np.arange(N) / (N * dk)
    t1, t2 = 0.9, 0.12
    ph = _ph(x, rho=np.full(N, 1.0 / N), t1=t1, t2=t2)
    alphas = rng.uniform(0.2, 2.8, P)
    phis = rng.uniform(0, 2 * math.pi, P)
    gx = dk / (GAMMA_BAR * tau)
    ev = make_events([(tau, gx, 0, 0, a, p, 1, 0.0) for a, p in zip(alphas, phis)])
    sig, _ = sim(ph, ev, GAMMA_BAR)
    ref = epg_signal(alphas, phis, tau, t1, t2, orders=P + 2)
    _close(sig, ref, 1e-12, "EPG (K-t) cross-check")


def pin_demodulation_phase(sim):
    """RF phase φ with receiver phase φ gives the same signal as φ = 0 (RF-spoiling reading)."""
    rng = np.random.default_rng(18)
    n = 6
    ph = _ph(rng.uniform(-0.2, 0.2, n), rho=rng.uniform(0.2, 1, n), t2=rng.uniform(0.02, 0.2, n),
             dw=2 * math.pi * rng.uniform(-100, 100, n))
    base = [(1e-3, 1e-3, 0, 0, 0, 0, 1, 0.0)] * 8
    s0, _ = sim(ph, make_events([(0.0, 0, 0, 0, 0.6, 0.0, 0, 0.0)] + base), GAMMA_BAR)
    for phi in (0.4, 2.0, 5.5):
        rows = [(0.0, 0, 0, 0, 0.6, phi, 0, 0.0)] + [r[:7] + (phi,) for r in base]
        s1, _ = sim(ph, make_events(rows), GAMMA_BAR)
        _close(s1, s0, 1e-14, "demodulation phase invariance")


def pin_invariants(sim):
    """Linearity in ρ, additivity over spin subsets (domain decomposition, §5.3.2), permutation."""
    from paper_1305_6861_gb300.workloads import random_phantom, random_sequence

    rng = np.random.default_rng(19)
    ph = random_phantom(40, rng)
    seq = random_sequence(120, rng)
    g = seq.gamma_hz_per_t
    s, _ = sim(ph, seq.events, g)
    ph2 = ph.subset(np.arange(ph.n))
    ph2.rho = ph2.rho * 2.5
    s2, _ = sim(ph2, seq.events, g)
    _close(s2, 2.5 * s, 1e-13, "linearity in rho")
    a, b = ph.subset(np.arange(0, 17)), ph.subset(np.arange(17, 40))
    sa, _ = sim(a, seq.events, g)
    sb, _ = sim(b, seq.events, g)
    _close(sa + sb, s, 1e-13, "additivity over spin subsets")
    perm = rng.permutation(ph.n)
    sp, _ = sim(ph.subset(perm), seq.events, g)
    _close(sp, s, 1e-13, "permutation invariance")


def pin_degenerate(sim):
    """Zero spins → zero signal; zero events; Δt = 0 without RF is the identity; T = ∞ never decays."""
    from paper_1305_6861_gb300.workloads import random_sequence

    seq = random_sequence(30, np.random.default_rng(20))
    empty = _ph(np.zeros(0))
    s, _ = sim(empty, seq.events, GAMMA_BAR)
    assert s.shape == (seq.n_adc,) and not np.any(s), "empty phantom must give a zero signal"
    ph = _ph([0.1], rho=[0.5])
    m0 = np.array([[0.2, -0.3, 0.1]])
    _, st = sim(ph, make_events([]), GAMMA_BAR, m_init=m0, want_signal=False, want_state=True)
    _close(st, m0, 0.0, "no events")
    _, st = sim(ph, make_events([(0.0, 1e-2, 0, 0, 0, 0, 0, 0.0)] * 3), GAMMA_BAR, m_init=m0, want_signal=False, want_state=True)
    _close(st, m0, 0.0, "zero-length events")
    _, st = sim(ph, make_events([(10.0, 0, 0, 0, 0, 0, 0, 0.0)]), GAMMA_BAR, m_init=m0, want_signal=False, want_state=True)
    _close(st, m0, 1e-15, "T = inf")


ALL_PINS = [
    pin_rf_rotation,
    pin_special_flips,
    pin_free_precession_expm,
    pin_bruteforce_sequences,
    pin_fid,
    pin_t1_recovery,
    pin_spin_echo,
    pin_worked_example_4_6,
    pin_imaging_equation,
    pin_epg_cross_check,
    pin_demodulation_phase,
    pin_invariants,
    pin_degenerate,
]
