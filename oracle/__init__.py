"""The oracle: TEST INFRASTRUCTURE ONLY.

A plain C reference of the paper's first-level J/psi event selection
(arXiv:1810.11966, Sec. 3.2) plus its CHAIN-mode extension, used to check the
GPU library.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import it.  It shares no code with the GPU path; the
only thing both sides use is the seeded input generator in ``synth``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jpsi_oracle.c")
_HDR = os.path.join(_HERE, "jpsi_oracle.h")
_LIB = os.path.join(_HERE, "libjpsi_oracle.so")

OK, EINVAL, ENOMEM, ECAPACITY = 0, 1, 2, 3
MODE_PAPER, MODE_CHAIN = 0, 1


class Params(ctypes.Structure):
    _fields_ = [
        ("n_stations", ctypes.c_int32),
        ("trigger_station", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("ndf", ctypes.c_int32),
        ("min_candidates", ctypes.c_int32),
        ("t_xz", ctypes.c_float),
        ("t_yz", ctypes.c_float),
        ("distinct_hits", ctypes.c_int32),
    ]


class Stream(ctypes.Structure):
    _fields_ = [("n_windows", ctypes.c_int32), ("dt", ctypes.c_float), ("bounds", ctypes.c_void_p)]


def params(n_stations=4, mode=MODE_CHAIN, t_xz=0.25, t_yz=None, ndf=2, min_candidates=2, trigger_station=None,
           distinct_hits=0):
    p = Params()
    p.distinct_hits = distinct_hits
    p.n_stations = n_stations
    p.trigger_station = n_stations - 1 if trigger_station is None else trigger_station
    p.mode = mode
    p.ndf = ndf
    p.min_candidates = min_candidates
    p.t_xz = t_xz
    p.t_yz = t_xz if t_yz is None else t_yz
    return p


def build(force: bool = False) -> str:
    """Compile the oracle: -O2 with FP contraction off, so a*b+c is never fused."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        lib.jpsi_oracle_run.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, ctypes.c_int64, vp, vp, vp, vp,
                                        vp, vp, vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int]
        lib.jpsi_oracle_run.restype = ctypes.c_int
        f3 = ctypes.c_float * 3
        lib.jpsi_oracle_triplet.argtypes = [f3, f3, f3, ctypes.c_float, ctypes.c_float, vp, vp, vp, vp]
        lib.jpsi_oracle_triplet.restype = ctypes.c_int
        lib.jpsi_oracle_triplet64.argtypes = [f3, f3, f3, ctypes.c_double, ctypes.c_double, vp, vp, vp, vp]
        lib.jpsi_oracle_triplet64.restype = ctypes.c_int
        lib.jpsi_oracle_cut.argtypes = [ctypes.c_int32, ctypes.c_float]
        lib.jpsi_oracle_cut.restype = ctypes.c_float
        lib.jpsi_oracle_stream.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Stream), ctypes.c_int64, vp, vp, vp,
                                           vp, vp, vp, vp, vp, vp, ctypes.c_int64, vp, vp]
        lib.jpsi_oracle_stream.restype = ctypes.c_int
        _lib = lib
    return _lib


def cut(ndf: int, t: float) -> float:
    return _load().jpsi_oracle_cut(ndf, t)


def triplet(xs, ys, zs, c_xz, c_yz, fp64=False):
    """P1 on one triplet.  Returns (pass, m_x, m_y, S_x, S_y)."""
    lib = _load()
    f3 = ctypes.c_float * 3
    if fp64:
        v = [ctypes.c_double() for _ in range(4)]
        ok = lib.jpsi_oracle_triplet64(f3(*xs), f3(*ys), f3(*zs), c_xz, c_yz, *[ctypes.addressof(a) for a in v])
    else:
        v = [ctypes.c_float() for _ in range(4)]
        ok = lib.jpsi_oracle_triplet(f3(*xs), f3(*ys), f3(*zs), c_xz, c_yz, *[ctypes.addressof(a) for a in v])
    return (bool(ok),) + tuple(a.value for a in v)


def run(p: Params, batch, *, triplets=True, capacity=None, n_threads=1, brute=False, fp64=False):
    """Runs the oracle over a host batch (dict with x, y, z, offsets, n_events).

    Returns dict(status, accept_bits, track_counts, unit_counts, trip_off,
    triplets [n,3] int32 or None, trip_needed).
    """
    lib = _load()
    n_ev = int(batch["n_events"])
    S = p.n_stations
    x = np.ascontiguousarray(batch["x"], dtype=np.float32)
    y = np.ascontiguousarray(batch["y"], dtype=np.float32)
    z = np.ascontiguousarray(batch["z"], dtype=np.float32)
    off = np.ascontiguousarray(batch["offsets"], dtype=np.int32)
    n_hits = int(batch.get("n_hits", x.size))
    acc = np.zeros((n_ev + 31) // 32, np.uint32)
    tc = np.zeros(n_ev, np.int32)
    uc = np.zeros(n_ev * S, np.int32)
    to = np.zeros(n_ev * S + 1, np.int64)
    needed = ctypes.c_int64(-1)
    if triplets:
        if capacity is None:
            # size from a counting run first (two-pass, like the GPU library)
            rc = lib.jpsi_oracle_run(ctypes.byref(p), n_ev, n_hits, x.ctypes.data, y.ctypes.data, z.ctypes.data,
                                     off.ctypes.data if off.size else None, None, None, None, None, 0,
                                     ctypes.byref(needed), None, n_threads, int(brute), int(fp64))
            if rc != OK:
                return {"status": rc}
            capacity = needed.value
        trip = np.zeros((max(int(capacity), 1), 3), np.int32)
        tptr = trip.ctypes.data
    else:
        trip, tptr = None, None
    rc = lib.jpsi_oracle_run(ctypes.byref(p), n_ev, n_hits, x.ctypes.data, y.ctypes.data, z.ctypes.data,
                             off.ctypes.data if off.size else None, acc.ctypes.data, tc.ctypes.data,
                             to.ctypes.data, tptr, int(capacity or 0), ctypes.byref(needed), uc.ctypes.data,
                             n_threads, int(brute), int(fp64))
    res = {"status": rc, "accept_bits": acc, "track_counts": tc, "unit_counts": uc, "trip_off": to,
           "trip_needed": needed.value}
    if triplets and rc == OK:
        res["triplets"] = trip[: needed.value]
    else:
        res["triplets"] = None
    return res


def stream(p: Params, ts, bounds, dt, *, triplets=True):
    """The free-streaming selection over one timeslice (dict with x, y, z, t
    and offsets [n_stations*3 + 1], each layer group sorted by t): windows
    [bounds[k], bounds[k+1]), coincidence width dt.  Returns the dict of
    run() with windows in place of events."""
    lib = _load()
    S = p.n_stations
    b = np.ascontiguousarray(bounds, dtype=np.float32)
    K = len(b) - 1
    x, y, z, t = (np.ascontiguousarray(ts[k], dtype=np.float32) for k in ("x", "y", "z", "t"))
    off = np.ascontiguousarray(ts["offsets"], dtype=np.int32)
    sp = Stream(K, dt, b.ctypes.data)
    acc = np.zeros((K + 31) // 32, np.uint32)
    tc = np.zeros(K, np.int32)
    uc = np.zeros(K * S, np.int32)
    to = np.zeros(K * S + 1, np.int64)
    needed = ctypes.c_int64(-1)
    args = [ctypes.byref(p), ctypes.byref(sp), x.size, x.ctypes.data, y.ctypes.data, z.ctypes.data, t.ctypes.data,
            off.ctypes.data]
    rc = lib.jpsi_oracle_stream(*args, acc.ctypes.data, tc.ctypes.data, to.ctypes.data, None, 0,
                                ctypes.byref(needed), uc.ctypes.data)
    res = {"status": rc, "accept_bits": acc, "track_counts": tc, "unit_counts": uc, "trip_off": to,
           "trip_needed": needed.value, "triplets": None}
    if rc == OK and triplets:
        trip = np.zeros((max(needed.value, 1), 3), np.int32)
        rc = lib.jpsi_oracle_stream(*args, acc.ctypes.data, tc.ctypes.data, to.ctypes.data, trip.ctypes.data,
                                    needed.value, ctypes.byref(needed), uc.ctypes.data)
        res["status"] = rc
        res["triplets"] = trip[: needed.value]
    return res
