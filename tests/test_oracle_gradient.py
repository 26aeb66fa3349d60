"""The oracle's forward-mode gradient against central finite differences of the oracle forward
and against an exact identity (the signal is linear in M0 for fixed T1/T2)."""
import math

import numpy as np
import pytest

from paper_1305_6861_gb300 import workloads as W


def _case(seed, n_sp=6, n_rf=12):
    rng = np.random.default_rng(seed)
    ph = W.random_phantom(n_sp, rng, inf_frac=0.0)
    ph.t1[:] = rng.uniform(0.2, 1.5, n_sp)
    ph.t2[:] = np.minimum(rng.uniform(0.02, 0.2, n_sp), ph.t1)
    # shaped excitation with learnable sub-pulses, then a short readout, repeated 3 times
    base = W.sinc_pulse(0.5, n_rf, 4.0)
    rows, params = [], []
    for tr in range(3):
        for i, a in enumerate(base):
            rows.append((20e-6, 0, 0, 2e-3, float(a), 0.3 * tr, 0, 0.0))
            params.append(i)
        rows.append((1e-3, -1e-3, 2e-3 * (tr - 1), 0, 0, 0, 0, 0.0))
        rows += [(20e-6, 2e-3, 0, 0, 0, 0, 1, 0.3 * tr)] * 8
        params += [-1] * 9
        rows.append((4e-3, 0, 0, 0, 0, 0, 0, 0.0))
        params.append(-1)
    ev = W.make_events(rows)
    rf = np.array(base) * rng.uniform(0.8, 1.2, n_rf)
    return ph, ev, np.array(params, dtype=np.int32), rf, rng


def _loss(oracle_mod, ph, ev, params, rf, target):
    s = oracle_mod.simulate_rf(ph, ev, W.GAMMA_BAR, params, rf)
    return float(np.sum(np.abs(s - target) ** 2)), s


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(oracle_mod, seed):
    ph, ev, params, rf, rng = _case(seed)
    target = oracle_mod.simulate_rf(ph, ev, W.GAMMA_BAR, params, rf * 1.1) * 0.9
    L0, s = _loss(oracle_mod, ph, ev, params, rf, target)
    h = 2 * (s - target)  # dL/dRe s + j dL/dIm s for L = |s - t|^2
    sel = [0, 3, 5, 11]
    g_rho, g_t1, g_t2, g_rf = oracle_mod.gradient(ph, ev, W.GAMMA_BAR, h, params, rf, sel)
    eps = 1e-4
    for name, arr, grad in (("rho", ph.rho, g_rho), ("t1", ph.t1, g_t1), ("t2", ph.t2, g_t2)):
        for k in range(ph.n):
            step = eps * abs(arr[k])  # relative step: T2 can be 0.02 s
            old = arr[k]
            arr[k] = old + step
            lp, _ = _loss(oracle_mod, ph, ev, params, rf, target)
            arr[k] = old - step
            lm, _ = _loss(oracle_mod, ph, ev, params, rf, target)
            arr[k] = old
            fd = (lp - lm) / (2 * step)
            assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)), (name, k, fd, grad[k])
    for i, p in enumerate(sel):
        rp, rm = rf.copy(), rf.copy()
        step = eps * max(abs(rf[p]), 1e-3)
        rp[p] += step
        rm[p] -= step
        fd = (_loss(oracle_mod, ph, ev, params, rp, target)[0] - _loss(oracle_mod, ph, ev, params, rm, target)[0]) / (2 * step)
        assert abs(fd - g_rf[i]) <= 1e-6 * max(1.0, abs(fd)), (p, fd, g_rf[i])


def test_rho_gradient_exact_linearity(oracle_mod):
    """For a loss linear in the signal, L = Re(conj(h)·s), dL/dM0_s = L of spin s alone / M0_s."""
    ph, ev, params, rf, rng = _case(7)
    n_adc = int(np.count_nonzero(ev["adc"]))
    h = rng.normal(size=n_adc) + 1j * rng.normal(size=n_adc)
    g_rho, _, _, _ = oracle_mod.gradient(ph, ev, W.GAMMA_BAR, h, params, rf)
    for k in range(ph.n):
        one = ph.subset([k])
        s = oracle_mod.simulate_rf(one, ev, W.GAMMA_BAR, params, rf)
        want = float(np.real(np.sum(np.conj(h) * s))) / ph.rho[k]
        assert abs(g_rho[k] - want) <= 1e-12 * max(1.0, abs(want))
