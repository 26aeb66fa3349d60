"""Test-side interpreter of the compiled float64 device program (host-compiler check, no GPU).

It executes the operation stream that ``mrsim_debug_compile`` returns with numpy, with the
semantics the kernels implement (pulse frame, lazy T1 per pulse, cached precession and T1
classes with explicit reloads, sample runs with anchors and leading inline precessions), so that the host compiler's
rewrites — merged intervals, fused sub-pulses, frame tracking, class selection, cache
bookkeeping, run grouping — can be compared with the oracle on the CPU.  It is test
infrastructure, not a fallback: the library never calls it.
"""
import math

import numpy as np

from paper_1305_6861_gb300 import mrsim as M


def interpret(events, gamma, ph, state_in=None, snapshots=None):
    """Returns (signal, final state, ops[, snapshots]); snapshots: the states (laboratory frame)
    after the given event indices, when asked for."""
    prog = M.debug_compile(events, gamma, snapshots=snapshots)
    ops, pcls, e1tab, e2tab, demod, train = (prog[k] for k in ("ops", "pcls", "e1", "e2", "demod", "train"))
    n_adc = demod.shape[0]
    x, y, z, rho = ph.x, ph.y, ph.z, ph.rho
    df = ph.dw / (2 * math.pi)
    with np.errstate(divide="ignore"):
        r1 = np.where(np.isinf(ph.t1), 0.0, 1.0 / ph.t1)
        r2 = np.where(np.isinf(ph.t2), 0.0, 1.0 / ph.t2)
    W = [np.exp(-c[3] * r2) * np.exp(-2j * math.pi * (c[0] * x + c[1] * y + c[2] * z + df * c[3])) for c in pcls]
    E1 = [-np.expm1(-t * r1) for t in e1tab]
    E2 = [np.exp(-t * r2) for t in e2tab]
    adc_phase = events["adc_phase"][events["adc"] != 0]
    sig = np.zeros(n_adc, dtype=complex)
    if state_in is None:
        m = np.zeros(ph.n, dtype=complex)  # u + jv in the pulse frame (ψ = 0 at the start)
        mz = rho.copy()
    else:
        m = state_in[:, 0] + 1j * state_in[:, 1]
        mz = state_in[:, 2].copy()
    psi = 0.0  # frame angle, tracked here independently from the ops' frame turns
    snaps = np.zeros((0 if snapshots is None else len(snapshots), ph.n, 3))
    wc = None  # register caches of the kernel
    e1c = None

    def sample(j, v):
        # lab frame: Mx + jMy = (u + jv)·e^{jψ}; demodulate by e^{-j adc_phase}; the table the
        # kernel uses must be exactly that factor
        want = np.exp(1j * psi) * np.exp(-1j * adc_phase[j])
        assert abs(demod[j] - want) < 1e-12, (j, demod[j], want)
        sig[j] += v.sum() * demod[j]

    def t1(op):
        nonlocal mz, e1c
        if op["flags"] & M.F_E1CLS:
            if op["flags"] & M.F_E1LOAD:
                e1c = E1[op["ecls"]]
            mz = mz - e1c * (mz - rho)
        elif op["flags"] & M.F_E1INL:
            mz = mz - (-np.expm1(-op["f"][10] * r1)) * (mz - rho)

    def pcls_use(op):
        nonlocal wc
        if op["flags"] & M.F_PLOAD:
            wc = W[op["pcls"]]
        return wc

    def inline(op):
        f = op["f"]
        e2 = E2[op["ecls"]] if op["flags"] & M.F_E2CLS else np.exp(-f[3] * r2)
        th = f[0] * x + f[1] * y + f[2] * z + f[3] * df
        return e2 * np.exp(-2j * math.pi * th)

    for op in ops:
        k, fl, f = op["kind"], op["flags"], op["f"]
        if k == M.OP_RF_TRAIN:
            w = wc
            for ca, sa in train[op["adc0"] : op["adc0"] + op["n"]]:
                mz = mz - e1c * (mz - rho)
                v = m.imag
                nv = ca * v + sa * mz
                mz = ca * mz - sa * v
                m = (m.real + 1j * nv) * w
            continue
        if k in (M.OP_RF, M.OP_RF_FAST):
            if fl & M.F_FRAME:
                d = math.atan2(f[3], f[2])
                m = m * np.exp(-1j * d)
                psi += d
            if k == M.OP_RF_FAST:
                mz = mz - e1c * (mz - rho)
            else:
                t1(op)
            ca, sa = f[0], f[1]
            v = m.imag
            nv = ca * v + sa * mz
            mz = ca * mz - sa * v
            m = m.real + 1j * nv
            if k == M.OP_RF_FAST or fl & M.F_PCLS:
                m = m * pcls_use(op)
            if fl & M.F_ADC:
                sample(op["adc0"], m)
        elif k == M.OP_PREC:
            if fl & M.F_PCLS:
                for _ in range(op["n"]):
                    m = m * pcls_use(op)
            elif fl & M.F_INLINE:
                m = m * inline(op)
            if fl & M.F_ADC:
                sample(op["adc0"], m)
        elif k == M.OP_RUN:
            start = m  # the anchor restores from the state before the run's own precession
            if fl & M.F_INLINE:
                m = m * inline(op)
            w = pcls_use(op)
            for t in range(op["n"]):
                m = m * w
                sample(op["adc0"] + t, m)
            if fl & M.F_ANCHOR:
                m = start * W[op["acls"]]
        elif k == M.OP_SNAP:
            t1(op)
            assert abs(math.atan2(f[1], f[0]) - math.atan2(math.sin(psi), math.cos(psi))) < 1e-9
            lab = m * (f[0] + 1j * f[1])
            snaps[op["adc0"]] = np.stack([lab.real, lab.imag, mz], 1)
        else:
            t1(op)
            assert abs(math.atan2(f[1], f[0]) - math.atan2(math.sin(psi), math.cos(psi))) < 1e-9
    lab = m * np.exp(1j * psi)
    state = np.stack([lab.real, lab.imag, mz], 1)
    if snapshots is not None:
        return sig, state, ops, snaps
    return sig, state, ops
