"""Python binding of libjpsi, the GB300 (sm_103a) first-level J/psi event
selection of arXiv:1810.11966 (Sec. 3.2) with its CHAIN-mode extension.

Argument marshalling only: every step of the selection runs in the CUDA
library (include/jpsi.h).  The functions carry the names of the C entry
points; ``Context`` and ``select`` are conveniences that allocate the output
tensors with PyTorch.  There is no CPU fallback: if the library cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# JPSI_LIBRARY may name another build of the library, e.g. libjpsi_checked.so
# (bounds-checked stores) beside this file
LIB_PATH = os.environ.get("JPSI_LIBRARY") or os.path.join(_HERE, "libjpsi.so")

JPSI_OK, JPSI_EINVAL, JPSI_ENOMEM, JPSI_ECAPACITY, JPSI_ECUDA, JPSI_ETIMEOUT, JPSI_EBUSY = range(7)
JPSI_MODE_PAPER, JPSI_MODE_CHAIN = 0, 1

# every symbol include/jpsi.h declares
EXPORTS = ("jpsi_create", "jpsi_destroy", "jpsi_run_plain", "jpsi_run", "jpsi_run_host", "jpsi_autotune",
           "jpsi_serve_start", "jpsi_serve_submit", "jpsi_serve_wait", "jpsi_serve_stop", "jpsi_strerror",
           "jpsi_last_error", "jpsi_timing_enable", "jpsi_timing_get", "jpsi_select_noalloc", "jpsi_get_tuning",
           "jpsi_set_tuning", "jpsi_run_stream", "jpsi_run_stream_plain", "jpsi_inject_fault")
FAULT_ALLOC, FAULT_RUN = 1, 2


class JpsiError(RuntimeError):
    def __init__(self, status, detail=""):
        self.status = status
        super().__init__(f"{_strerror(status)} ({status}){': ' + detail if detail else ''}")


class jpsi_params(ctypes.Structure):
    _fields_ = [("n_stations", ctypes.c_int32), ("trigger_station", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("ndf", ctypes.c_int32), ("min_candidates", ctypes.c_int32), ("t_xz", ctypes.c_float),
                ("t_yz", ctypes.c_float), ("distinct_hits", ctypes.c_int32)]


class jpsi_batch(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_int64), ("n_hits", ctypes.c_int64), ("x", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("z", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("z_layer", ctypes.c_void_p)]


class jpsi_outputs(ctypes.Structure):
    _fields_ = [("accept_bits", ctypes.c_void_p), ("track_counts", ctypes.c_void_p), ("trip_off", ctypes.c_void_p),
                ("triplets", ctypes.c_void_p), ("trip_capacity", ctypes.c_int64), ("trip_needed", ctypes.c_int64)]


class jpsi_timeslice(ctypes.Structure):
    _fields_ = [("n_hits", ctypes.c_int64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("t", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("z_layer", ctypes.c_void_p),
                ("n_windows", ctypes.c_int64), ("bounds", ctypes.c_void_p), ("dt", ctypes.c_float)]


class jpsi_timing(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("light_ms", ctypes.c_double),
                ("count_rest_ms", ctypes.c_double), ("emit_ms", ctypes.c_double),
                ("light_wpb", ctypes.c_int32), ("light_grab", ctypes.c_int32), ("window_ms", ctypes.c_double)]


class jpsi_tuning(ctypes.Structure):
    _fields_ = [("light_wpb", ctypes.c_int32), ("light_grab", ctypes.c_int32), ("small_layer_cap", ctypes.c_int32),
                ("medium_layer_cap", ctypes.c_int32), ("heavy_ctas_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("record_cap", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_lib = None


def load(build_if_missing: bool = False):
    """Loads libjpsi.so (building it first when asked).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _b
        _b.build()
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libjpsi.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, vp = ctypes.POINTER, ctypes.c_void_p
    st = ctypes.c_int
    lib.jpsi_create.argtypes = [P(jpsi_params), ctypes.c_int, ctypes.c_size_t, P(vp)]
    lib.jpsi_create.restype = st
    lib.jpsi_destroy.argtypes = [vp]
    lib.jpsi_destroy.restype = None
    for name in ("jpsi_run_plain", "jpsi_run", "jpsi_run_host"):
        f = getattr(lib, name)
        f.argtypes = [vp, P(jpsi_batch), P(jpsi_outputs), vp]
        f.restype = st
    for name in ("jpsi_run_stream", "jpsi_run_stream_plain"):
        f = getattr(lib, name)
        f.argtypes = [vp, P(jpsi_timeslice), P(jpsi_outputs), vp]
        f.restype = st
    lib.jpsi_autotune.argtypes = [vp, P(jpsi_batch)]
    lib.jpsi_autotune.restype = st
    lib.jpsi_serve_start.argtypes = [vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
    lib.jpsi_serve_start.restype = st
    lib.jpsi_serve_submit.argtypes = [vp, P(jpsi_batch), P(jpsi_outputs), P(ctypes.c_uint64)]
    lib.jpsi_serve_submit.restype = st
    lib.jpsi_serve_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_double)]
    lib.jpsi_serve_wait.restype = st
    lib.jpsi_serve_stop.argtypes = [vp]
    lib.jpsi_serve_stop.restype = st
    lib.jpsi_strerror.argtypes = [ctypes.c_int]
    lib.jpsi_strerror.restype = ctypes.c_char_p
    lib.jpsi_last_error.argtypes = [vp]
    lib.jpsi_last_error.restype = ctypes.c_char_p
    lib.jpsi_timing_enable.argtypes = [vp, ctypes.c_int]
    lib.jpsi_timing_enable.restype = st
    lib.jpsi_timing_get.argtypes = [vp, P(jpsi_timing)]
    lib.jpsi_timing_get.restype = st
    lib.jpsi_inject_fault.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.jpsi_inject_fault.restype = st
    lib.jpsi_select_noalloc.argtypes = [P(jpsi_params), P(jpsi_batch), vp, vp, vp]
    lib.jpsi_select_noalloc.restype = st
    lib.jpsi_get_tuning.argtypes = [vp, P(jpsi_tuning)]
    lib.jpsi_get_tuning.restype = st
    lib.jpsi_set_tuning.argtypes = [vp, P(jpsi_tuning)]
    lib.jpsi_set_tuning.restype = st
    _lib = lib
    return lib


def _strerror(status):
    try:
        return load().jpsi_strerror(status).decode()
    except Exception:
        return "status"


# ------------------------------------------------------------ C entry points

def jpsi_create(params: jpsi_params, device: int = 0, hbm_budget: int = 0):
    ctx = ctypes.c_void_p()
    s = load().jpsi_create(ctypes.byref(params), device, hbm_budget, ctypes.byref(ctx))
    if s != JPSI_OK:
        raise JpsiError(s, "jpsi_create")
    return ctx


def jpsi_destroy(ctx):
    load().jpsi_destroy(ctx)


def jpsi_last_error(ctx) -> str:
    return load().jpsi_last_error(ctx).decode()


def jpsi_strerror(status: int) -> str:
    return load().jpsi_strerror(status).decode()


def jpsi_run_plain(ctx, batch: jpsi_batch, out: jpsi_outputs, stream=0) -> int:
    return load().jpsi_run_plain(ctx, ctypes.byref(batch), ctypes.byref(out), stream)


def jpsi_run(ctx, batch: jpsi_batch, out: jpsi_outputs, stream=0) -> int:
    return load().jpsi_run(ctx, ctypes.byref(batch), ctypes.byref(out), stream)


def jpsi_run_host(ctx, batch: jpsi_batch, out: jpsi_outputs, stream=0) -> int:
    return load().jpsi_run_host(ctx, ctypes.byref(batch), ctypes.byref(out), stream)


def jpsi_run_stream(ctx, ts: jpsi_timeslice, out: jpsi_outputs, stream=0) -> int:
    return load().jpsi_run_stream(ctx, ctypes.byref(ts), ctypes.byref(out), stream)


def jpsi_run_stream_plain(ctx, ts: jpsi_timeslice, out: jpsi_outputs, stream=0) -> int:
    return load().jpsi_run_stream_plain(ctx, ctypes.byref(ts), ctypes.byref(out), stream)


def jpsi_autotune(ctx, sample: jpsi_batch) -> int:
    return load().jpsi_autotune(ctx, ctypes.byref(sample))


def jpsi_serve_start(ctx, n_slots, slot_events, slot_hits, slot_triplets) -> int:
    return load().jpsi_serve_start(ctx, n_slots, slot_events, slot_hits, slot_triplets)


def jpsi_serve_submit(ctx, batch: jpsi_batch, out: jpsi_outputs):
    t = ctypes.c_uint64()
    s = load().jpsi_serve_submit(ctx, ctypes.byref(batch), ctypes.byref(out), ctypes.byref(t))
    return s, t.value


def jpsi_serve_wait(ctx, ticket, timeout_ms=-1):
    r, lat = ctypes.c_int(), ctypes.c_double()
    s = load().jpsi_serve_wait(ctx, ticket, timeout_ms, ctypes.byref(r), ctypes.byref(lat))
    return s, r.value, lat.value


def jpsi_serve_stop(ctx) -> int:
    return load().jpsi_serve_stop(ctx)


def jpsi_timing_enable(ctx, enable=True) -> int:
    return load().jpsi_timing_enable(ctx, int(enable))


def jpsi_timing_get(ctx) -> jpsi_timing:
    t = jpsi_timing()
    s = load().jpsi_timing_get(ctx, ctypes.byref(t))
    if s != JPSI_OK:
        raise JpsiError(s, "jpsi_timing_get")
    return t


def jpsi_inject_fault(ctx, kind: int, count: int) -> int:
    """Host-side fault injection for tests (FAULT_ALLOC or FAULT_RUN)."""
    return load().jpsi_inject_fault(ctx, kind, count)


def jpsi_get_tuning(ctx) -> jpsi_tuning:
    t = jpsi_tuning()
    s = load().jpsi_get_tuning(ctx, ctypes.byref(t))
    if s != JPSI_OK:
        raise JpsiError(s, "jpsi_get_tuning")
    return t


def jpsi_set_tuning(ctx, t: jpsi_tuning) -> int:
    return load().jpsi_set_tuning(ctx, ctypes.byref(t))


def jpsi_select_noalloc(params: jpsi_params, batch: jpsi_batch, track_counts, unit_counts, stream=0) -> int:
    """Counting without allocation (see include/jpsi.h): device pointers for
    track_counts [n_events] and unit_counts [n_events * n_stations]."""
    return load().jpsi_select_noalloc(ctypes.byref(params), ctypes.byref(batch), track_counts, unit_counts, stream)


# --------------------------------------------------------------- helpers

def params(n_stations=4, mode=JPSI_MODE_CHAIN, t_xz=0.25, t_yz=None, ndf=2, min_candidates=2,
           trigger_station=None, distinct_hits=0) -> jpsi_params:
    p = jpsi_params()
    p.distinct_hits = distinct_hits
    p.n_stations = n_stations
    p.trigger_station = n_stations - 1 if trigger_station is None else trigger_station
    p.mode = mode
    p.ndf = ndf
    p.min_candidates = min_candidates
    p.t_xz = t_xz
    p.t_yz = t_xz if t_yz is None else t_yz
    return p


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr() if a.numel() else None
    return a.ctypes.data if a.size else None


def make_batch(x, y, z, offsets, n_events=None, n_hits=None, z_layer=None) -> jpsi_batch:
    """A jpsi_batch over torch tensors (device) or numpy arrays (host).  z may
    be None when z_layer (n_stations * 3 floats, same memory kind) is given."""
    b = jpsi_batch()
    nev = n_events if n_events is not None else (len(offsets) - 1) // 3
    b.n_events = int(nev)
    b.n_hits = int(n_hits if n_hits is not None else len(x))
    b.x, b.y, b.offsets = _ptr(x), _ptr(y), _ptr(offsets)
    b.z = None if z is None else _ptr(z)
    b.z_layer = None if z_layer is None else _ptr(z_layer)
    return b


def make_timeslice(x, y, z, t, offsets, bounds, dt, z_layer=None) -> jpsi_timeslice:
    """A jpsi_timeslice over device tensors: hits grouped per (station, layer)
    with offsets [3S+1], each group sorted by t; windows from bounds [K+1]."""
    ts = jpsi_timeslice()
    ts.n_hits = int(len(x))
    ts.x, ts.y, ts.t, ts.offsets = _ptr(x), _ptr(y), _ptr(t), _ptr(offsets)
    ts.z = None if z is None else _ptr(z)
    ts.z_layer = None if z_layer is None else _ptr(z_layer)
    ts.n_windows = max(int(len(bounds)) - 1, 0)
    ts.bounds = _ptr(bounds)
    ts.dt = float(dt)
    return ts


class Context:
    """Owns a jpsi context; ``select`` allocates outputs as torch tensors."""

    def __init__(self, p: jpsi_params, device: int = 0, hbm_budget: int = 0):
        load()
        self.p = p
        self.device = device
        self.ctx = jpsi_create(p, device, hbm_budget)

    def close(self):
        if self.ctx:
            jpsi_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self):
        return jpsi_last_error(self.ctx)

    def check(self, s):
        if s != JPSI_OK:
            raise JpsiError(s, self.last_error())

    def select_stream(self, x, y, z, t, offsets, bounds, dt, *, triplets=True, capacity=None, form="batched",
                      stream=None, z_layer=None):
        """Free-streaming selection of one timeslice (device tensors): windows
        [bounds[k], bounds[k+1]) in place of events.  Returns what ``select``
        returns; triplet rows index the timeslice's layer groups."""
        ts = make_timeslice(x, y, z, t, offsets, bounds, dt, z_layer=z_layer)
        run = {"batched": jpsi_run_stream, "plain": jpsi_run_stream_plain}[form]
        return self._outputs(lambda o, st: run(self.ctx, ts, o, st), int(ts.n_windows), triplets, capacity, stream)

    def select(self, x, y, z, offsets, n_events, *, triplets=True, capacity=None, form="batched", stream=None,
               z_layer=None):
        """Runs the selection on device tensors.  Returns a dict with the run's
        status and the device tensors accept_bits, track_counts, trip_off,
        triplets ([n,3]) and trip_needed (statuses are returned, not
        raised).  With capacity=None the call sizes the triplet buffer from a
        first counting run (two calls, like the library's own two-pass
        contract).  z may be None with a per-layer table z_layer (device)."""
        b = make_batch(x, y, z, offsets, n_events, z_layer=z_layer)
        run = {"batched": jpsi_run, "plain": jpsi_run_plain}[form]
        return self._outputs(lambda o, st: run(self.ctx, b, o, st), n_events, triplets, capacity, stream)

    def _outputs(self, call, n_events, triplets, capacity, stream):
        import torch
        dev = torch.device("cuda", self.device)
        S = self.p.n_stations
        nu = n_events * S
        out = {
            "accept_bits": torch.empty(max((n_events + 31) // 32, 1), dtype=torch.int32, device=dev),
            "track_counts": torch.empty(max(n_events, 1), dtype=torch.int32, device=dev),
            "trip_off": torch.empty(nu + 1, dtype=torch.int64, device=dev),
        }
        o = jpsi_outputs()
        o.accept_bits = out["accept_bits"].data_ptr()
        o.track_counts = out["track_counts"].data_ptr()
        o.trip_off = out["trip_off"].data_ptr()
        st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        tr = None
        if triplets:
            if capacity is None:
                s = call(o, st)
                if s != JPSI_OK:
                    out.update(status=s, trip_needed=o.trip_needed, triplets=None, error=self.last_error())
                    return out
                capacity = o.trip_needed
            tr = torch.empty((max(capacity, 1), 3), dtype=torch.int32, device=dev)
            o.triplets = tr.data_ptr()
            o.trip_capacity = capacity
        s = call(o, st)
        out["status"] = s
        out["error"] = self.last_error() if s != JPSI_OK else ""
        out["trip_needed"] = o.trip_needed
        out["triplets"] = tr[: o.trip_needed] if (triplets and s == JPSI_OK) else None
        out["accept_bits"] = out["accept_bits"][: (n_events + 31) // 32]
        out["track_counts"] = out["track_counts"][:n_events]
        return out
