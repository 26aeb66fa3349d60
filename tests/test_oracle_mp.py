"""High-precision pins of the oracle (mpmath, 40 significant digits) on one to three spins.

The reference here is the Bloch equation itself: for piecewise-constant fields each event is the
exponential of the augmented generator of Eqs. A.1-A.4 (free precession and relaxation) and of
the rotating-frame B1 generator of Eq. A.12 (the hard pulse), evaluated with mpmath's matrix
exponential — no closed form of the oracle is reused.  The gradient reference is mpmath's
numerical differentiation of that solution with respect to M0, T1, T2 and the learnable flip
angles, at a precision where its error is far below float64.  So the float64 oracle must match
to its own rounding (measured ~1e-15), and its forward-mode gradient to 1e-12 (measured
~5e-15; the float64 central differences of the other gradient test only reach 1e-6)."""
import math

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W

mp = pytest.importorskip("mpmath")
DPS = 40


def _free_gen(gamma, bz, t1, t2, m0):
    r1 = mp.mpf(0) if t1 == mp.inf else 1 / t1
    r2 = mp.mpf(0) if t2 == mp.inf else 1 / t2
    A = mp.zeros(4, 4)
    A[0, 0] = -r2
    A[0, 1] = gamma * bz
    A[1, 0] = -gamma * bz
    A[1, 1] = -r2
    A[2, 2] = -r1
    A[2, 3] = m0 * r1
    return A


def _rf_gen(phi):
    s, c = mp.sin(phi), mp.cos(phi)
    K = mp.zeros(4, 4)
    K[0, 2] = -s
    K[1, 2] = c
    K[2, 0] = s
    K[2, 1] = -c
    return K


def mp_signal(spins, events, gamma_hz, flips):
    """Complex samples (mpc) of the summed spins; spins: tuples (x, y, z, m0, t1, t2, dw) of mpf,
    flips: the flip angle of every event (mpf)."""
    gamma = 2 * mp.pi * mp.mpf(gamma_hz)
    n_adc = int(np.count_nonzero(events["adc"]))
    sig = [mp.mpc(0)] * n_adc
    for x, y, z, m0, t1, t2, dw in spins:
        v = mp.matrix([0, 0, m0, 1])
        j = 0
        for e, alpha in zip(events, flips):
            if alpha != 0:
                v = mp.expm(alpha * _rf_gen(mp.mpf(float(e["rf_phase"])))) * v
            bz = mp.mpf(float(e["gx"])) * x + mp.mpf(float(e["gy"])) * y + mp.mpf(float(e["gz"])) * z + dw / gamma
            v = mp.expm(mp.mpf(float(e["dt"])) * _free_gen(gamma, bz, t1, t2, m0)) * v
            if e["adc"]:
                sig[j] += mp.mpc(v[0], v[1]) * mp.expj(-mp.mpf(float(e["adc_phase"])))
                j += 1
    return sig


def _mp_spins(ph):
    f = lambda a: mp.inf if math.isinf(a) else mp.mpf(float(a))
    return [tuple(f(getattr(ph, k)[s]) for k in ("x", "y", "z", "rho", "t1", "t2", "dw")) for s in range(ph.n)]


def _moderate_sequence(rng, n_tr=3, n_read=5):
    """Pulses of any flip/phase, encodings, readouts and rests with phases of at most a few tens
    of rad per event (so the float64 oracle's own rounding stays near 1e-15)."""
    rows = []
    for tr in range(n_tr):
        rows.append((rng.uniform(0, 1e-3), 0, 0, 1e-3, rng.uniform(-2, 2), rng.uniform(0, 2 * math.pi), 0, 0.0))
        rows.append((1e-3, *(rng.normal(size=3) * 1e-3), 0, 0, 0, 0.0))
        for _ in range(n_read):
            rows.append((2e-5, 2e-3, 0, 0, 0, 0, 1, rng.uniform(0, 2 * math.pi)))
        rows.append((rng.uniform(1e-3, 5e-3), 0, 0, 0, 0, 0, 0, 0.0))
    return W.make_events(rows)


@pytest.mark.parametrize("seed", range(3))
def test_oracle_matches_high_precision_bloch_solution(oracle_mod, seed):
    rng = np.random.default_rng(900 + seed)
    n = 1 + seed  # one to three spins
    ph = W.random_phantom(n, rng, fov=0.2, inf_frac=0.2)
    ph.dw[:] = 2 * math.pi * rng.uniform(-100, 100, n)
    ev = _moderate_sequence(rng)
    with mp.workdps(DPS):
        ref = mp_signal(_mp_spins(ph), ev, W.GAMMA_BAR, [mp.mpf(float(a)) for a in ev["rf_flip"]])
        ref = np.array([complex(s) for s in ref])
    got = oracle_mod.simulate(ph, ev, W.GAMMA_BAR)[0]
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_oracle_gradient_matches_high_precision_derivatives(oracle_mod):
    rng = np.random.default_rng(77)
    ph = W.random_phantom(2, rng, fov=0.2, inf_frac=0.0)
    ph.t1[:] = rng.uniform(0.2, 1.0, 2)
    ph.t2[:] = np.minimum(rng.uniform(0.02, 0.1, 2), ph.t1)
    ph.dw[:] = 2 * math.pi * rng.uniform(-80, 80, 2)
    n_rf = 4
    rows, params = [], []
    for tr in range(2):
        for i in range(n_rf):  # a shaped excitation: learnable sub-pulses
            rows.append((2e-5, 0, 0, 2e-3, 0.2, 0.4 * tr, 0, 0.0))
            params.append(i)
        rows.append((1e-3, -1e-3, 1e-3 * tr, 0, 0, 0, 0, 0.0))
        rows += [(2e-5, 2e-3, 0, 0, 0, 0, 1, 0.4 * tr)] * 4
        rows.append((3e-3, 0, 0, 0, 0, 0, 0, 0.0))
        params += [-1] * 6
    ev = W.make_events(rows)
    params = np.array(params, dtype=np.int32)
    rf = rng.uniform(0.1, 0.5, n_rf)
    n_adc = int(ev["adc"].sum())
    h = rng.normal(size=n_adc) + 1j * rng.normal(size=n_adc)
    g_rho, g_t1, g_t2, g_rf = oracle_mod.gradient(ph, ev, W.GAMMA_BAR, h, params, rf, list(range(n_rf)))

    with mp.workdps(DPS):
        spins = _mp_spins(ph)
        rf_mp = [mp.mpf(float(a)) for a in rf]
        hm = [mp.mpc(float(c.real), float(c.imag)) for c in h]

        def loss(spins_, rf_):
            flips = [rf_[p] if p >= 0 else mp.mpf(float(a)) for p, a in zip(params, ev["rf_flip"])]
            s = mp_signal(spins_, ev, W.GAMMA_BAR, flips)
            return mp.fsum(mp.re(mp.conj(hc) * sc) for hc, sc in zip(hm, s))  # dL/ds = h

        def d_spin(s, k):
            def f(v):
                sp = [list(t) for t in spins]
                sp[s][k] = v
                return loss([tuple(t) for t in sp], rf_mp)
            return float(mp.diff(f, spins[s][k]))

        def d_rf(i):
            def f(v):
                r = list(rf_mp)
                r[i] = v
                return loss(spins, r)
            return float(mp.diff(f, rf_mp[i]))

        ref_rho = [d_spin(s, 3) for s in range(ph.n)]
        ref_t1 = [d_spin(s, 4) for s in range(ph.n)]
        ref_t2 = [d_spin(s, 5) for s in range(ph.n)]
        ref_rf = [d_rf(i) for i in range(n_rf)]

    for got, ref in ((g_rho, ref_rho), (g_t1, ref_t1), (g_t2, ref_t2), (g_rf, ref_rf)):
        ref = np.asarray(ref)
        assert np.max(np.abs(np.asarray(got) - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref))), (got, ref)
