"""Thin ctypes binding of libmrsim (include/mrsim.h).

Argument marshalling only: every step of the simulation runs in the CUDA library.
There is no CPU fallback — if ``lib/libmrsim.so`` is missing or no sm_103 GPU is
present, the calls raise.  Arrays may be numpy arrays (host) or CUDA tensors
(anything with ``data_ptr()`` and ``is_cuda``); streams are ``cudaStream_t``
handles as integers (e.g. ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os
from enum import IntEnum

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmrsim.so")

FP64 = 0
FP32 = 1
FP32_KAHAN = 2  # the float32 path with its float64 cross-block sums (same results as FP32)
ACCUMULATE = 1
TUNE = 2

EVENT_DTYPE = np.dtype(
    [("dt", "<f8"), ("gx", "<f8"), ("gy", "<f8"), ("gz", "<f8"), ("rf_flip", "<f8"),
     ("rf_phase", "<f8"), ("adc_phase", "<f8"), ("adc", "<i4"), ("reserved", "<i4")]
)

# Every symbol include/mrsim.h declares (checked by the CPU tests).
EXPORTS = (
    "mrsim_status_string", "mrsim_last_error", "mrsim_context_create", "mrsim_context_destroy",
    "mrsim_stream_status", "mrsim_phantom_create", "mrsim_phantom_create_device", "mrsim_phantom_num_spins",
    "mrsim_phantom_destroy", "mrsim_sequence_load", "mrsim_sequence_num_adc", "mrsim_sequence_num_events",
    "mrsim_sequence_num_ops", "mrsim_sequence_destroy", "mrsim_simulate", "mrsim_simulate_ex",
    "mrsim_simulate_coils", "mrsim_kt_simulate", "mrsim_max_config_k", "mrsim_sequence_load_snapshots",
    "mrsim_sequence_num_snapshots", "mrsim_debug_compile_snapshots",
    "mrsim_debug_compile", "mrsim_autotune", "mrsim_batch_create", "mrsim_batch_num_items",
    "mrsim_batch_autotune", "mrsim_batch_set_shape", "mrsim_batch_launch", "mrsim_batch_launch_graph",
    "mrsim_batch_destroy", "mrsim_simulate_batch", "mrsim_simulate_batch_static",
    "mrsim_adjoint_create", "mrsim_adjoint_num_adc", "mrsim_adjoint_forward", "mrsim_adjoint_backward",
    "mrsim_adjoint_destroy", "mrsim_compile", "mrsim_compile_last_error", "mrsim_compiled_num_adc",
    "mrsim_compiled_upload_bytes", "mrsim_compiled_destroy", "mrsim_sequence_create", "mrsim_debug_wait_timeout",
    "mrsim_set_log_callback", "mrsim_debug_fail_alloc", "mrsim_measure_fma_rate", "mrsim_simulate_adjoint",
    "mrsim_sequence_num_pulses", "mrsim_simulate_fields", "mrsim_phantom_set_b0_direction", "mrsim_fields_create",
    "mrsim_fields_num_adc", "mrsim_fields_destroy", "mrsim_adjoint_set_precision", "mrsim_context_set_train_maps",
    "mrsim_fields_num_train_maps",
)


class Status(IntEnum):
    OK = 0
    EINVAL = 1
    ENOMEM = 2
    ECUDA = 3
    ETIMEOUT = 4
    EUNSUPPORTED = 5


class MrsimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{Status(status).name}: {msg}")
        self.status = Status(status)


class ProgramDump(ctypes.Structure):
    _fields_ = [
        ("ops", ctypes.c_void_p), ("n_ops", ctypes.c_int64),
        ("pcls", ctypes.c_void_p), ("n_pcls", ctypes.c_int32), ("n_e1", ctypes.c_int32),
        ("e1", ctypes.c_void_p), ("e2", ctypes.c_void_p), ("n_e2", ctypes.c_int32), ("n_train", ctypes.c_int32),
        ("train", ctypes.c_void_p), ("demod", ctypes.c_void_p), ("n_adc", ctypes.c_int64),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("spins_per_thread", ctypes.c_int32),
        ("threads_per_block", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("reserved", ctypes.c_int32),
        ("state_in", ctypes.c_void_p),
        ("state_out", ctypes.c_void_p),
        ("snapshots", ctypes.c_void_p),
    ]


_lib = None


def lib():
    """The loaded library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "mrsim_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "mrsim_last_error": (ctypes.c_char_p, [vp]),
            "mrsim_context_create": (ctypes.c_int, [ctypes.c_int, P(vp)]),
            "mrsim_context_destroy": (None, [vp]),
            "mrsim_stream_status": (ctypes.c_int, [vp, vp]),
            "mrsim_phantom_create": (ctypes.c_int, [vp, i64] + [vp] * 7 + [P(vp)]),
            "mrsim_phantom_create_device": (ctypes.c_int, [vp, i64] + [vp] * 7 + [vp, P(vp)]),
            "mrsim_phantom_num_spins": (i64, [vp]),
            "mrsim_phantom_destroy": (None, [vp]),
            "mrsim_sequence_load": (ctypes.c_int, [vp, i64, vp, dbl, P(vp)]),
            "mrsim_sequence_num_adc": (i64, [vp]),
            "mrsim_sequence_num_events": (i64, [vp]),
            "mrsim_sequence_num_ops": (i64, [vp]),
            "mrsim_sequence_destroy": (None, [vp]),
            "mrsim_simulate": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp, vp, i64]),
            "mrsim_simulate_ex": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp, vp, i64, P(Options)]),
            "mrsim_autotune": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp, P(Options)]),
            "mrsim_simulate_coils": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp, i32, vp, vp, i64]),
            "mrsim_kt_simulate": (ctypes.c_int, [vp, i64, vp, vp, vp, vp, i64, vp, i32, ctypes.c_int, vp, vp, i64]),
            "mrsim_max_config_k": (ctypes.c_int, [i64, vp, ctypes.c_double, vp]),
            "mrsim_sequence_load_snapshots": (ctypes.c_int, [vp, i64, vp, ctypes.c_double, i64, vp, P(vp)]),
            "mrsim_sequence_num_snapshots": (i64, [vp]),
            "mrsim_debug_compile_snapshots": (ctypes.c_int, [i64, vp, ctypes.c_double, i64, vp, P(ProgramDump)]),
            "mrsim_batch_create": (ctypes.c_int, [vp, i32, vp, vp, ctypes.c_int, vp, P(vp)]),
            "mrsim_batch_num_items": (i64, [vp]),
            "mrsim_batch_autotune": (ctypes.c_int, [vp, vp, P(Options)]),
            "mrsim_batch_set_shape": (ctypes.c_int, [vp, i32, i32]),
            "mrsim_batch_launch": (ctypes.c_int, [vp, vp]),
            "mrsim_batch_launch_graph": (ctypes.c_int, [vp, vp]),
            "mrsim_batch_destroy": (None, [vp]),
            "mrsim_simulate_batch": (ctypes.c_int, [vp, i32, vp, vp, ctypes.c_int, vp, vp]),
            "mrsim_simulate_batch_static": (ctypes.c_int, [vp, i32, vp, vp, ctypes.c_int, vp, vp, i32, i32]),
            "mrsim_adjoint_create": (ctypes.c_int, [vp, i64, vp, dbl, vp, i32, i32, P(vp)]),
            "mrsim_adjoint_num_adc": (i64, [vp]),
            "mrsim_adjoint_forward": (ctypes.c_int, [vp, vp, vp, vp, vp]),
            "mrsim_adjoint_backward": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "mrsim_adjoint_destroy": (None, [vp]),
            "mrsim_adjoint_set_precision": (ctypes.c_int, [vp, ctypes.c_int]),
            "mrsim_simulate_adjoint": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, i32, vp, vp, vp, vp, vp, vp]),
            "mrsim_sequence_num_pulses": (i64, [vp]),
            "mrsim_simulate_fields": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp, vp, i64]),
            "mrsim_phantom_set_b0_direction": (ctypes.c_int, [vp, vp, vp]),
            "mrsim_fields_create": (ctypes.c_int, [vp, i64, vp, vp, dbl, dbl, P(vp)]),
            "mrsim_fields_num_adc": (i64, [vp]),
            "mrsim_fields_num_train_maps": (i32, [vp]),
            "mrsim_fields_destroy": (None, [vp]),
            "mrsim_debug_compile": (ctypes.c_int, [i64, vp, dbl, P(ProgramDump)]),
            "mrsim_compile": (ctypes.c_int, [i64, vp, dbl, i64, vp, P(vp)]),
            "mrsim_compile_last_error": (ctypes.c_char_p, []),
            "mrsim_compiled_num_adc": (i64, [vp]),
            "mrsim_compiled_upload_bytes": (i64, [vp]),
            "mrsim_compiled_destroy": (None, [vp]),
            "mrsim_sequence_create": (ctypes.c_int, [vp, vp, P(vp)]),
            "mrsim_debug_wait_timeout": (ctypes.c_int, [vp, i64, vp]),
            "mrsim_set_log_callback": (None, [vp, vp]),
            "mrsim_debug_fail_alloc": (ctypes.c_int, [vp, i32]),
            "mrsim_context_set_train_maps": (ctypes.c_int, [vp, i32]),
            "mrsim_measure_fma_rate": (ctypes.c_int, [vp, i32, dbl, vp, P(dbl), P(dbl)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    """Raw address of a numpy array or CUDA tensor (None → NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


class Context:
    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        rc = lib().mrsim_context_create(int(device), ctypes.byref(h))
        if rc != 0:
            raise MrsimError(rc, f"mrsim_context_create(device={device}) failed")
        self.h = h

    def check(self, rc):
        if rc != 0:
            raise MrsimError(rc, lib().mrsim_last_error(self.h).decode())

    def stream_status(self, stream=None):
        self.check(lib().mrsim_stream_status(self.h, _stream(stream)))

    def set_train_maps(self, enable: bool):
        """Recurring shaped pulses as one map per spin (default) or sub-pulse by sub-pulse."""
        self.check(lib().mrsim_context_set_train_maps(self.h, 1 if enable else 0))

    def close(self):
        if getattr(self, "h", None):
            lib().mrsim_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Phantom:
    """Spin list on the device.  `arrays` = (x, y, z, rho, t1, t2, dw), float64, host or CUDA."""

    def __init__(self, ctx: Context, arrays, stream=None):
        self.ctx = ctx
        arrs = list(arrays)
        n = int(arrs[0].shape[0])
        h = ctypes.c_void_p()
        if hasattr(arrs[0], "is_cuda") and arrs[0].is_cuda:
            rc = lib().mrsim_phantom_create_device(ctx.h, n, *[_ptr(a) for a in arrs], _stream(stream), ctypes.byref(h))
        else:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
            self._keep = arrs
            rc = lib().mrsim_phantom_create(ctx.h, n, *[_ptr(a) for a in arrs], ctypes.byref(h))
        ctx.check(rc)
        self.h = h
        self.n = n

    @classmethod
    def from_workload_phantom(cls, ctx, ph, stream=None):
        return cls(ctx, ph.arrays(), stream)

    def close(self):
        if getattr(self, "h", None):
            lib().mrsim_phantom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Compiled:
    """Host-compiled program (mrsim_compile): no context and no GPU involved, so it can be built on
    a worker thread while a context simulates (ctypes releases the GIL during the call)."""

    def __init__(self, events, gamma_hz_per_t: float, snapshots=None):
        ev = np.ascontiguousarray(events)
        if ev.dtype != EVENT_DTYPE:
            ev = ev.astype(EVENT_DTYPE)
        sn = np.ascontiguousarray([] if snapshots is None else snapshots, dtype=np.int64)
        h = ctypes.c_void_p()
        rc = lib().mrsim_compile(ev.shape[0], _ptr(ev), float(gamma_hz_per_t), sn.shape[0],
                                 _ptr(sn) if sn.shape[0] else None, ctypes.byref(h))
        if rc != 0:
            raise MrsimError(rc, lib().mrsim_compile_last_error().decode())
        self.h = h
        self.n_adc = int(lib().mrsim_compiled_num_adc(h))
        self.upload_bytes = int(lib().mrsim_compiled_upload_bytes(h))

    def close(self):
        if getattr(self, "h", None):
            lib().mrsim_compiled_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sequence:
    """Compiled event list (host numpy array of EVENT_DTYPE records)."""

    def __init__(self, ctx: Context, events, gamma_hz_per_t: float, snapshots=None):
        """`snapshots`: event indices after which every spin's state is recorded (§7.2)."""
        self.ctx = ctx
        ev = np.ascontiguousarray(events)
        if ev.dtype != EVENT_DTYPE:
            ev = ev.astype(EVENT_DTYPE)
        h = ctypes.c_void_p()
        if snapshots is None:
            ctx.check(lib().mrsim_sequence_load(ctx.h, ev.shape[0], _ptr(ev), float(gamma_hz_per_t), ctypes.byref(h)))
        else:
            sn = np.ascontiguousarray(snapshots, dtype=np.int64)
            ctx.check(lib().mrsim_sequence_load_snapshots(ctx.h, ev.shape[0], _ptr(ev), float(gamma_hz_per_t),
                                                          sn.shape[0], _ptr(sn), ctypes.byref(h)))
        self.h = h
        self.n_snapshots = int(lib().mrsim_sequence_num_snapshots(h))
        self.n_adc = int(lib().mrsim_sequence_num_adc(h))
        self.n_events = int(lib().mrsim_sequence_num_events(h))
        self.n_ops = int(lib().mrsim_sequence_num_ops(h))

    @classmethod
    def from_workload_sequence(cls, ctx, seq):
        return cls(ctx, seq.events, seq.gamma_hz_per_t)

    @classmethod
    def from_compiled(cls, ctx: Context, compiled: "Compiled"):
        """Upload a host-compiled program (mrsim_sequence_create)."""
        self = cls.__new__(cls)
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx.check(lib().mrsim_sequence_create(ctx.h, compiled.h, ctypes.byref(h)))
        self.h = h
        self.n_snapshots = int(lib().mrsim_sequence_num_snapshots(h))
        self.n_adc = int(lib().mrsim_sequence_num_adc(h))
        self.n_events = int(lib().mrsim_sequence_num_events(h))
        self.n_ops = int(lib().mrsim_sequence_num_ops(h))
        return self

    def close(self):
        if getattr(self, "h", None):
            lib().mrsim_sequence_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate(ctx: Context, phantom: Phantom, seq: Sequence, precision: int = FP32, stream=None, out=None,
             spins_per_thread: int = 0, threads_per_block: int = 0, accumulate: bool = False,
             state_in=None, state_out=None, snapshots=None):
    """Run the forward simulation.  `out`: numpy complex128[n_adc] (host, returned when None) or a CUDA
    buffer of 2*n_adc float64 (asynchronous on `stream`)."""
    if out is None:
        out = np.zeros(seq.n_adc, dtype=np.complex128)
    opt = Options(int(spins_per_thread), int(threads_per_block), ACCUMULATE if accumulate else 0, 0,
                  _ptr(state_in), _ptr(state_out), _ptr(snapshots))
    rc = lib().mrsim_simulate_ex(ctx.h, phantom.h, seq.h, int(precision), _stream(stream), _ptr(out), seq.n_adc,
                                 ctypes.byref(opt))
    ctx.check(rc)
    return out


MAX_COILS = 8


def simulate_coils(ctx: Context, phantom: Phantom, seq: Sequence, sens, precision: int = FP32, stream=None,
                   out=None):
    """Receive-coil signals: `sens` complex [n_coils, n_spins] (numpy complex128, or a CUDA buffer of
    n_coils*2*n_spins float64 with `n_coils` taken from its length).  `out`: numpy complex128
    [n_coils, n_adc] (host, returned when None) or a CUDA buffer of n_coils*2*n_adc float64."""
    if isinstance(sens, np.ndarray):
        sens = np.ascontiguousarray(sens, dtype=np.complex128)
        if sens.ndim != 2 or sens.shape[1] != phantom.n:
            raise ValueError("sens must be [n_coils, n_spins]")
        n_coils = sens.shape[0]
    else:
        n_coils = int(sens.numel()) // max(2 * phantom.n, 1)
    if out is None:
        out = np.zeros((n_coils, seq.n_adc), dtype=np.complex128)
    rc = lib().mrsim_simulate_coils(ctx.h, phantom.h, seq.h, int(precision), _stream(stream), int(n_coils),
                                    _ptr(sens), _ptr(out), seq.n_adc)
    ctx.check(rc)
    return out


KT_MAX_ORDER = 255


def max_config_k(events, gamma_hz_per_t: float) -> np.ndarray:
    """Largest |k| [rad/m] per axis that any configuration of the event list reaches (Eq. 5.1)."""
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    out = np.zeros(3)
    rc = lib().mrsim_max_config_k(ev.shape[0], _ptr(ev), float(gamma_hz_per_t), _ptr(out))
    if rc != 0:
        raise MrsimError(rc, "mrsim_max_config_k failed")
    return out


def delta_x_max(events, gamma_hz_per_t: float) -> np.ndarray:
    """Largest isochromat spacing per axis free of aliasing, Δx_max = π / K_max (Eq. 5.2); inf where
    no configuration moves along the axis."""
    k = max_config_k(events, gamma_hz_per_t)
    with np.errstate(divide="ignore"):
        return np.where(k > 0, np.pi / np.where(k > 0, k, 1.0), np.inf)


def kt_simulate(ctx: Context, t1, t2, steps, max_order: int, b1=None, df=None, precision: int = FP32,
                stream=None, out=None):
    """K-t formalism (§4.2) for n ensembles: t1, t2 [s], b1 (flip scale), df [Hz] as float64 numpy
    arrays or CUDA tensors; `steps`: workloads.KT_STEP_DTYPE array.  Returns (or fills) the
    ensembles' samples: numpy complex128 [n, n_samples] or a CUDA buffer of n*2*n_samples float64."""
    from . import workloads as W

    st = np.ascontiguousarray(steps, dtype=W.KT_STEP_DTYPE)
    n_samples = int(np.count_nonzero(st["sample"]))

    def arr(a):
        if a is None or hasattr(a, "data_ptr"):
            return a
        return np.ascontiguousarray(a, dtype=np.float64)

    t1, t2, b1, df = arr(t1), arr(t2), arr(b1), arr(df)
    n = int(t1.shape[0]) if hasattr(t1, "shape") else int(t1.numel())
    if out is None:
        out = np.zeros((n, n_samples), dtype=np.complex128)
    rc = lib().mrsim_kt_simulate(ctx.h, n, _ptr(t1), _ptr(t2), _ptr(b1), _ptr(df), st.shape[0], _ptr(st),
                                 int(max_order), int(precision), _stream(stream), _ptr(out), n_samples)
    ctx.check(rc)
    return out


class Batch:
    """Many phantom/sequence pairs in one persistent launch.  `outs`: one CUDA buffer of 2*n_adc
    float64 per pair (e.g. torch tensors); phantoms and sequences must outlive the batch."""

    def __init__(self, ctx: Context, phantoms, seqs, precision: int = FP32, outs=None):
        self.ctx = ctx
        self._keep = (list(phantoms), list(seqs), list(outs))
        n = len(self._keep[0])
        ph = (ctypes.c_void_p * n)(*[p.h.value for p in phantoms])
        sq = (ctypes.c_void_p * n)(*[q.h.value for q in seqs])
        os_ = (ctypes.c_void_p * n)(*[_ptr(o).value for o in outs])
        self._arrays = (ph, sq, os_)
        h = ctypes.c_void_p()
        ctx.check(lib().mrsim_batch_create(ctx.h, n, ph, sq, int(precision), os_, ctypes.byref(h)))
        self.h = h

    @property
    def n_items(self) -> int:
        return int(lib().mrsim_batch_num_items(self.h))

    def autotune(self, stream=None):
        opt = Options()
        self.ctx.check(lib().mrsim_batch_autotune(self.h, _stream(stream), ctypes.byref(opt)))
        return int(opt.spins_per_thread), int(opt.threads_per_block)

    def set_shape(self, spins_per_thread: int, threads_per_block: int):
        self.ctx.check(lib().mrsim_batch_set_shape(self.h, int(spins_per_thread), int(threads_per_block)))

    def launch(self, stream=None, graph: bool = False):
        f = lib().mrsim_batch_launch_graph if graph else lib().mrsim_batch_launch
        self.ctx.check(f(self.h, _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().mrsim_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate_batch_static(ctx: Context, phantoms, seqs, precision: int, outs, stream=None,
                          spins_per_thread: int = 0, threads_per_block: int = 0):
    """Batch launch that allocates no device memory (scratch in the library's fixed static array):
    for callers that cannot call cudaMalloc.  `outs`: one CUDA buffer of 2*n_adc float64 per pair
    (required; this call allocates none).  Asynchronous on `stream`; calls that overlap on the GPU
    share the scratch and must not overlap."""
    n = len(phantoms)
    if len(seqs) != n or len(outs) != n:
        raise ValueError(f"{n} phantoms, {len(seqs)} sequences and {len(outs)} outputs: the lengths must agree")
    ph = (ctypes.c_void_p * n)(*[p.h.value for p in phantoms])
    sq = (ctypes.c_void_p * n)(*[q.h.value for q in seqs])
    os_ = (ctypes.c_void_p * n)(*[_ptr(o).value for o in outs])
    ctx.check(lib().mrsim_simulate_batch_static(ctx.h, n, ph, sq, int(precision), _stream(stream), os_,
                                                int(spins_per_thread), int(threads_per_block)))


class Adjoint:
    """Compiled event list for differentiation (float64).  rf_param: None or one int per event
    (index of the learnable flip angle that event uses, -1 = its own flip)."""

    def __init__(self, ctx: Context, events, gamma_hz_per_t: float, rf_param=None, n_params: int = 0,
                 ckpt_every: int = 64):
        self.ctx = ctx
        ev = np.ascontiguousarray(events)
        if ev.dtype != EVENT_DTYPE:
            ev = ev.astype(EVENT_DTYPE)
        rp = None if rf_param is None else np.ascontiguousarray(rf_param, dtype=np.int32)
        self._keep = (ev, rp)
        h = ctypes.c_void_p()
        ctx.check(lib().mrsim_adjoint_create(ctx.h, ev.shape[0], _ptr(ev), float(gamma_hz_per_t), _ptr(rp),
                                             int(n_params), int(ckpt_every), ctypes.byref(h)))
        self.h = h
        self.n_params = int(n_params)
        self.n_adc = int(lib().mrsim_adjoint_num_adc(h))

    def set_precision(self, precision: int):
        """FP64 (default) or FP32_KAHAN (the recursion in double-float pairs on the FP32 pipe)."""
        self.ctx.check(lib().mrsim_adjoint_set_precision(self.h, int(precision)))

    def forward(self, phantom: Phantom, rf_values=None, out=None, stream=None):
        self.ctx.check(lib().mrsim_adjoint_forward(self.h, phantom.h, _ptr(rf_values), _stream(stream), _ptr(out)))
        return out

    def backward(self, phantom: Phantom, dl_dsignal, rf_values=None, d_rho=None, d_t1=None, d_t2=None, d_rf=None,
                 stream=None):
        self.ctx.check(lib().mrsim_adjoint_backward(self.h, phantom.h, _ptr(rf_values), _ptr(dl_dsignal),
                                                    _stream(stream), _ptr(d_rho), _ptr(d_t1), _ptr(d_t2), _ptr(d_rf)))

    def close(self):
        if getattr(self, "h", None):
            lib().mrsim_adjoint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate_adjoint(ctx: Context, phantom: Phantom, seq: Sequence, dl_dsignal, precision: int = FP64,
                     ckpt_every: int = 64, stream=None, outs=None, rf: bool = True):
    """One-shot gradients (mrsim_simulate_adjoint) of a loss with dL/ds = `dl_dsignal` (numpy
    complex128[n_adc] or a CUDA buffer of 2*n_adc float64).  Returns (dL/dM0, dL/dT1, dL/dT2,
    dL/dα per pulse in event order, or None without `rf`) as numpy arrays, or fills `outs`
    (four buffers, host or CUDA, any of them None)."""
    if isinstance(dl_dsignal, np.ndarray):
        dl_dsignal = np.ascontiguousarray(dl_dsignal, dtype=np.complex128)
    if outs is None:
        n_p = int(lib().mrsim_sequence_num_pulses(seq.h))
        outs = [np.zeros(phantom.n), np.zeros(phantom.n), np.zeros(phantom.n), np.zeros(n_p) if rf else None]
    ctx.check(lib().mrsim_simulate_adjoint(ctx.h, phantom.h, seq.h, int(precision), int(ckpt_every), _ptr(dl_dsignal),
                                           _stream(stream), *[_ptr(o) for o in outs]))
    return tuple(outs)


def set_b0_direction(ctx: Context, phantom: Phantom, b0_dir, stream=None):
    """Static-field direction per spin (mrsim_phantom_set_b0_direction): [n_spins, 3] unit vectors,
    numpy or a CUDA buffer of 3*n_spins float64."""
    if isinstance(b0_dir, np.ndarray):
        b0_dir = np.ascontiguousarray(b0_dir, dtype=np.float64).reshape(-1)
    ctx.check(lib().mrsim_phantom_set_b0_direction(phantom.h, _ptr(b0_dir), _stream(stream)))


class Fields:
    """An event list prepared for non-parallel fields (mrsim_fields_create): g_transverse None or
    [n_events, 6] (gtx, gty) [T/m], b0_tesla the main field."""

    def __init__(self, ctx: Context, events, gamma_hz_per_t: float, g_transverse=None, b0_tesla: float = 1.5):
        self.ctx = ctx
        ev = np.ascontiguousarray(events)
        if ev.dtype != EVENT_DTYPE:
            ev = ev.astype(EVENT_DTYPE)
        gt = None if g_transverse is None else np.ascontiguousarray(g_transverse, dtype=np.float64).reshape(-1)
        h = ctypes.c_void_p()
        ctx.check(lib().mrsim_fields_create(ctx.h, ev.shape[0], _ptr(ev), _ptr(gt), float(gamma_hz_per_t),
                                            float(b0_tesla), ctypes.byref(h)))
        self.h = h
        self.n_adc = int(lib().mrsim_fields_num_adc(h))
        self.n_train_maps = int(lib().mrsim_fields_num_train_maps(h))
        self.n_events = int(ev.shape[0])

    def close(self):
        if getattr(self, "h", None):
            lib().mrsim_fields_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate_fields(ctx: Context, phantom: Phantom, fields: Fields, precision: int = FP32, stream=None, out=None):
    """Forward simulation with non-parallel fields (mrsim_simulate_fields).  Returns (or fills) the
    signal: numpy complex128[n_adc] or a CUDA buffer of 2*n_adc float64 (asynchronous)."""
    if out is None:
        out = np.zeros(fields.n_adc, dtype=np.complex128)
    ctx.check(lib().mrsim_simulate_fields(ctx.h, phantom.h, fields.h, int(precision), _stream(stream), _ptr(out),
                                          fields.n_adc))
    return out


def autotune(ctx: Context, phantom: Phantom, seq: Sequence, precision: int = FP32, stream=None):
    """Time every launch shape on a prefix of the program; the winner is kept in the sequence
    handle for this (precision, spin count).  Returns (spins_per_thread, threads_per_block)."""
    opt = Options()
    ctx.check(lib().mrsim_autotune(ctx.h, phantom.h, seq.h, int(precision), _stream(stream), ctypes.byref(opt)))
    return int(opt.spins_per_thread), int(opt.threads_per_block)


FMA_F32, FMA_F32X2, FMA_F64 = 0, 1, 2


def measure_fma_rate(ctx: Context, kind: int, target_ms: float = 100.0, stream=None):
    """Measured multiply-add rate of the device (mrsim_measure_fma_rate): (lane-ops/s, kernel ms)
    for kind FMA_F32, FMA_F32X2 or FMA_F64."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    ctx.check(lib().mrsim_measure_fma_rate(ctx.h, int(kind), float(target_ms), _stream(stream), ctypes.byref(rate),
                                           ctypes.byref(ms)))
    return rate.value, ms.value


def debug_compile(events, gamma_hz_per_t: float, snapshots=None):
    """Host-only compile of an event list (no GPU needed).  Returns a dict with the float64 device
    program (op records), the class tables, the sub-pulse table and the per-sample demodulation
    factors (complex)."""
    L = lib()
    ev = np.ascontiguousarray(events)
    if ev.dtype != EVENT_DTYPE:
        ev = ev.astype(EVENT_DTYPE)
    sn = np.ascontiguousarray([] if snapshots is None else snapshots, dtype=np.int64)

    def call(d):
        return L.mrsim_debug_compile_snapshots(ev.shape[0], _ptr(ev), float(gamma_hz_per_t), sn.shape[0],
                                               _ptr(sn) if sn.shape[0] else None, ctypes.byref(d))

    d = ProgramDump()
    rc = call(d)
    if rc != 0:
        raise MrsimError(rc, "mrsim_debug_compile failed")
    out = {
        "ops": np.zeros(d.n_ops, dtype=OP64_DTYPE),
        "pcls": np.zeros((d.n_pcls, 4)),
        "e1": np.zeros(d.n_e1),
        "e2": np.zeros(d.n_e2),
        "train": np.zeros((d.n_train, 2)),
        "demod": np.zeros(d.n_adc, dtype=np.complex128),
    }
    for f in ("ops", "pcls", "e1", "e2", "train", "demod"):
        setattr(d, f, out[f].ctypes.data)
    rc = call(d)
    if rc != 0:
        raise MrsimError(rc, "mrsim_debug_compile failed")
    return out


# Layout of one float64 device operation (128 bytes), for diagnostics.
OP64_DTYPE = np.dtype(
    [("kind", "u1"), ("rsv0", "u1"), ("flags", "<u2"), ("n", "<i4"), ("adc0", "<i4"), ("pcls", "<i2"),
     ("ecls", "<i2"), ("acls", "<i2"), ("tab", "<i2"), ("rsv2", "<i4"), ("f", "<f8", (13,))]
)
assert OP64_DTYPE.itemsize == 128
OP_END, OP_RF, OP_RF_FAST, OP_PREC, OP_RUN, OP_RF_TRAIN, OP_SNAP = 0, 1, 2, 3, 4, 5, 6
F_ADC, F_PCLS, F_PLOAD, F_INLINE, F_E1CLS, F_E1LOAD, F_E1INL, F_E2CLS, F_ANCHOR, F_FRAME = (
    1, 2, 4, 8, 16, 32, 64, 128, 256, 512)
F_KX, F_KY, F_KZ, F_DT = 1024, 2048, 4096, 8192
F_RFTAB, F_TMAP = 16384, 32768
