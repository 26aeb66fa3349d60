"""FP64 CPU oracle of the spin-based Bloch simulation (§5.1.1, Eq. 4.1).

TEST INFRASTRUCTURE ONLY: the reference that the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the library never does.  It shares no code with
the CUDA path: the arithmetic lives in ``mrsim_oracle.c`` (plain C, libm,
OpenMP over spins), this module only marshals arrays.

Inputs are plain numpy arrays (or any object with the seven phantom fields and
an ``events`` record array of 64-byte events); nothing here imports the
library package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrsim_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None

# Same byte layout as the library's event record (the interface, not shared code).
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
    ]
)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/lib/liboracle.so."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path):
    lib = ctypes.CDLL(path)
    d = ctypes.POINTER(ctypes.c_double)
    lib.oracle_simulate.restype = ctypes.c_int
    lib.oracle_simulate.argtypes = [ctypes.c_int64] + [d] * 7 + [d, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_double, d, ctypes.c_int64, d, ctypes.c_int]
    lib.oracle_max_threads.restype = ctypes.c_int
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_simulate_rf.restype = ctypes.c_int
    lib.oracle_simulate_rf.argtypes = [ctypes.c_int64] + [d] * 7 + [ctypes.c_int64, ctypes.c_void_p, ctypes.c_double,
                                       i32p, d, d, ctypes.c_int64, ctypes.c_int]
    lib.oracle_simulate_coils.restype = ctypes.c_int
    lib.oracle_simulate_coils.argtypes = [ctypes.c_int64] + [d] * 7 + [ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_double, ctypes.c_int32, d, d, ctypes.c_int64, ctypes.c_int]
    lib.oracle_simulate_fields.restype = ctypes.c_int
    lib.oracle_simulate_fields.argtypes = [ctypes.c_int64] + [d] * 7 + [d, ctypes.c_int64, ctypes.c_void_p, d,
                                           ctypes.c_double, ctypes.c_double, d, ctypes.c_int64, d, ctypes.c_int]
    lib.oracle_gradient.restype = ctypes.c_int
    lib.oracle_gradient.argtypes = [ctypes.c_int64] + [d] * 7 + [ctypes.c_int64, ctypes.c_void_p, ctypes.c_double,
                                    i32p, d, d, ctypes.c_int64, d, d, d, i32p, ctypes.c_int32, d, ctypes.c_int]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(_LIB)
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def simulate(phantom, events, gamma_hz_per_t, m_init=None, want_signal=True, want_state=False, n_threads=0, lib=None):
    """Run the oracle.  Returns (signal complex128[n_adc] or None, state float64[n,3] or None)."""
    lib = _load() if lib is None else lib
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    arrs = [np.ascontiguousarray(getattr(phantom, k), dtype=np.float64) for k in ("x", "y", "z", "rho", "t1", "t2", "dw")]
    n = arrs[0].shape[0]
    n_adc = int(np.count_nonzero(ev["adc"]))
    sig = np.zeros(2 * n_adc, dtype=np.float64) if want_signal else None
    st = np.zeros(3 * n, dtype=np.float64) if want_state else None
    mi = None
    if m_init is not None:
        mi = np.ascontiguousarray(np.asarray(m_init, dtype=np.float64).reshape(-1))
        if mi.shape[0] != 3 * n:
            raise ValueError("m_init must have 3 values per spin")
    rc = lib.oracle_simulate(
        n, *[_dp(a) for a in arrs], _dp(mi), ev.shape[0], ev.ctypes.data_as(ctypes.c_void_p),
        float(gamma_hz_per_t), _dp(sig), n_adc, _dp(st), int(n_threads)
    )
    if rc != 0:
        raise RuntimeError(f"oracle_simulate failed with code {rc}")
    out_sig = sig.view(np.complex128) if sig is not None else None
    out_st = st.reshape(n, 3) if st is not None else None
    return out_sig, out_st


def _ip(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def simulate_rf(phantom, events, gamma_hz_per_t, rf_param, rf_values, n_threads=0, lib=None):
    """Forward signal where event e's flip angle is rf_values[rf_param[e]] (rf_param[e] >= 0)."""
    lib = _load() if lib is None else lib
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    arrs = [np.ascontiguousarray(getattr(phantom, k), dtype=np.float64) for k in ("x", "y", "z", "rho", "t1", "t2", "dw")]
    rp = np.ascontiguousarray(rf_param, dtype=np.int32)
    rv = np.ascontiguousarray(rf_values, dtype=np.float64)
    n_adc = int(np.count_nonzero(ev["adc"]))
    sig = np.zeros(2 * n_adc)
    rc = lib.oracle_simulate_rf(arrs[0].shape[0], *[_dp(a) for a in arrs], ev.shape[0], ev.ctypes.data_as(ctypes.c_void_p),
                                float(gamma_hz_per_t), _ip(rp), _dp(rv), _dp(sig), n_adc, int(n_threads))
    if rc != 0:
        raise RuntimeError(f"oracle_simulate_rf failed with code {rc}")
    return sig.view(np.complex128)


def simulate_coils(phantom, events, gamma_hz_per_t, sens, n_threads=0, lib=None):
    """Receive-coil signals (Eq. 3.25 with per-spin sensitivities): sens is complex
    [n_coils, n_spins]; returns complex128 [n_coils, n_adc]."""
    lib = _load() if lib is None else lib
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    arrs = [np.ascontiguousarray(getattr(phantom, k), dtype=np.float64) for k in ("x", "y", "z", "rho", "t1", "t2", "dw")]
    n = arrs[0].shape[0]
    c = np.ascontiguousarray(np.asarray(sens, dtype=np.complex128))
    if c.ndim != 2 or c.shape[1] != n:
        raise ValueError("sens must be [n_coils, n_spins]")
    n_adc = int(np.count_nonzero(ev["adc"]))
    sig = np.zeros(2 * n_adc * c.shape[0])
    rc = lib.oracle_simulate_coils(n, *[_dp(a) for a in arrs], ev.shape[0], ev.ctypes.data_as(ctypes.c_void_p),
                                   float(gamma_hz_per_t), int(c.shape[0]), _dp(c.view(np.float64).reshape(-1)),
                                   _dp(sig), n_adc, int(n_threads))
    if rc != 0:
        raise RuntimeError(f"oracle_simulate_coils failed with code {rc}")
    return sig.view(np.complex128).reshape(c.shape[0], n_adc)


def simulate_fields(phantom, events, gamma_hz_per_t, ndir, gt=None, b0=1.5, want_state=False, n_threads=0,
                    lib=None):
    """Forward signal with non-parallel fields (§3.2, §3.4.3.2): ndir [n_spins, 3] unit static-field
    directions, gt None or [n_events, 6] transverse gradient components (gtx, gty) [T/m], b0 [T].
    Returns (signal complex128[n_adc], state [n, 3] or None)."""
    lib = _load() if lib is None else lib
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    arrs = [np.ascontiguousarray(getattr(phantom, k), dtype=np.float64) for k in ("x", "y", "z", "rho", "t1", "t2", "dw")]
    n = arrs[0].shape[0]
    nd = np.ascontiguousarray(np.asarray(ndir, dtype=np.float64).reshape(-1))
    if nd.shape[0] != 3 * n:
        raise ValueError("ndir must have 3 values per spin")
    g = None
    if gt is not None:
        g = np.ascontiguousarray(np.asarray(gt, dtype=np.float64).reshape(-1))
        if g.shape[0] != 6 * ev.shape[0]:
            raise ValueError("gt must have 6 values per event")
    n_adc = int(np.count_nonzero(ev["adc"]))
    sig = np.zeros(2 * n_adc)
    st = np.zeros(3 * n) if want_state else None
    rc = lib.oracle_simulate_fields(n, *[_dp(a) for a in arrs], _dp(nd), ev.shape[0], ev.ctypes.data_as(ctypes.c_void_p),
                                    _dp(g), float(gamma_hz_per_t), float(b0), _dp(sig), n_adc, _dp(st), int(n_threads))
    if rc != 0:
        raise RuntimeError(f"oracle_simulate_fields failed with code {rc}")
    return sig.view(np.complex128), (st.reshape(n, 3) if st is not None else None)


def gradient(phantom, events, gamma_hz_per_t, h, rf_param=None, rf_values=None, sel=(), n_threads=0, lib=None):
    """Forward-mode gradient of a loss whose gradient w.r.t. the signal is h (complex, per sample:
    dL/dRe s + j dL/dIm s).  Returns (dL/dM0, dL/dT1, dL/dT2 per spin, dL/d rf_values[sel])."""
    lib = _load() if lib is None else lib
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    arrs = [np.ascontiguousarray(getattr(phantom, k), dtype=np.float64) for k in ("x", "y", "z", "rho", "t1", "t2", "dw")]
    n = arrs[0].shape[0]
    hh = np.ascontiguousarray(np.asarray(h, dtype=np.complex128)).view(np.float64)
    n_adc = int(np.count_nonzero(ev["adc"]))
    if hh.shape[0] != 2 * n_adc:
        raise ValueError("h must have one complex value per sample")
    rp = None if rf_param is None else np.ascontiguousarray(rf_param, dtype=np.int32)
    rv = None if rf_values is None else np.ascontiguousarray(rf_values, dtype=np.float64)
    se = np.ascontiguousarray(np.asarray(sel, dtype=np.int32))
    out = [np.zeros(n) for _ in range(3)]
    dsel = np.zeros(max(len(se), 1))
    rc = lib.oracle_gradient(n, *[_dp(a) for a in arrs], ev.shape[0], ev.ctypes.data_as(ctypes.c_void_p),
                             float(gamma_hz_per_t), _ip(rp), _dp(rv), _dp(hh), n_adc, *[_dp(o) for o in out],
                             _ip(se) if len(se) else None, len(se), _dp(dsel), int(n_threads))
    if rc != 0:
        raise RuntimeError(f"oracle_gradient failed with code {rc}")
    return out[0], out[1], out[2], dsel[: len(se)]


def signal(workload_or_phantom, sequence=None, n_threads=0):
    """Convenience: complex signal of a workload (or phantom + sequence)."""
    if sequence is None:
        ph, seq = workload_or_phantom.phantom, workload_or_phantom.sequence
    else:
        ph, seq = workload_or_phantom, sequence
    s, _ = simulate(ph, seq.events, seq.gamma_hz_per_t, n_threads=n_threads)
    return s


class Variant:
    """The oracle compiled from another C source (used to check that the pins catch planted mistakes)."""

    def __init__(self, c_source: str, workdir: str):
        os.makedirs(workdir, exist_ok=True)
        src = os.path.join(workdir, "variant.c")
        so = os.path.join(workdir, "libvariant.so")
        with open(src, "w") as f:
            f.write(c_source)
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", so, src, "-lm"], check=True)
        self.lib = _bind(so)

    def simulate(self, *args, **kw):
        return simulate(*args, lib=self.lib, **kw)


def source() -> str:
    with open(_SRC) as f:
        return f.read()
