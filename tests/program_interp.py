"""Test-side interpreter of the compiled float64 device program (host-compiler check, no GPU).

It executes the operation stream that ``mrsim_debug_compile`` returns with numpy, with the
semantics the kernels implement (lazy T1 per pulse, cached precession classes, sample runs
with anchors), so that the host compiler's rewrites — merged intervals, fused sub-pulses,
class selection, run grouping — can be compared with the oracle on the CPU.  It is test
infrastructure, not a fallback: the library never calls it.
"""
import math

import numpy as np

from paper_1305_6861_gb300 import mrsim as M


def interpret(events, gamma, ph, state_in=None):
    ops, pcls, e1tab, e2tab, n_adc = M.debug_compile(events, gamma)
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
        mxy = np.zeros(ph.n, dtype=complex)
        dz = np.zeros(ph.n)
    else:
        mxy = state_in[:, 0] + 1j * state_in[:, 1]
        dz = state_in[:, 2] - rho

    def sample(j, v):
        sig[j] += v.sum() * np.exp(-1j * adc_phase[j])

    def t1(op):
        nonlocal dz
        if op["flags"] & M.F_E1CLS:
            dz = dz - E1[op["ecls"]] * dz
        elif op["flags"] & M.F_E1INL:
            dz = dz - (-np.expm1(-op["f"][10] * r1)) * dz

    for op in ops:
        k, fl, f = op["kind"], op["flags"], op["f"]
        if k == M.OP_RF:
            t1(op)
            R = f[:9].reshape(3, 3)
            v = np.stack([mxy.real, mxy.imag, dz + rho])
            nv = R @ v
            mxy = nv[0] + 1j * nv[1]
            dz = nv[2] - rho
            if fl & M.F_PCLS:
                mxy = mxy * W[op["pcls"]]
            if fl & M.F_ADC:
                sample(op["adc0"], mxy)
        elif k == M.OP_PREC:
            if fl & M.F_PCLS:
                for _ in range(op["n"]):
                    mxy = mxy * W[op["pcls"]]
            elif fl & M.F_INLINE:
                e2 = E2[op["ecls"]] if fl & M.F_E2CLS else np.exp(-f[3] * r2)
                th = f[0] * x + f[1] * y + f[2] * z + f[3] * df
                mxy = mxy * e2 * np.exp(-2j * math.pi * th)
            if fl & M.F_ADC:
                sample(op["adc0"], mxy)
        elif k == M.OP_RUN:
            start = mxy
            for t in range(op["n"]):
                mxy = mxy * W[op["pcls"]]
                sample(op["adc0"] + t, mxy)
            if fl & M.F_ANCHOR:
                mxy = start * W[op["acls"]]
        else:
            t1(op)
    state = np.stack([mxy.real, mxy.imag, dz + rho], 1)
    return sig, state, ops
