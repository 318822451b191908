"""Seeded synthetic event generator (input side only).

Shared by the test oracle and the GPU path; it holds none of the selection
arithmetic.  Events are shaped like the CBM muon-chamber events the paper
describes (Sec. 2: stations of three layers 10 cm apart; Sec. 3.1 and Fig. 2:
background hits around a central beam hole, signal muons as straight lines
from the target).  The paper's simulated data sets (Sec. 3.3, D1-D3) are not
available; these workloads stand in for them.

Every event is drawn from its own random streams, so ``generate(w, e0, n)``
returns exactly events ``e0 .. e0+n-1`` of the full workload.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jpsi_synth.c")
_LIB = os.path.join(_HERE, "libjpsi_synth.so")
MAX_STATIONS = 16


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("n_stations", ctypes.c_int32),
        ("radial", ctypes.c_int32),
        ("bg_mode", ctypes.c_int32),
        ("count_min", ctypes.c_int32),
        ("count_max", ctypes.c_int32),
        ("station_z", ctypes.c_double * MAX_STATIONS),
        ("layer_dz", ctypes.c_double),
        ("bg_lambda", ctypes.c_double),
        ("ln_median", ctypes.c_double),
        ("ln_sigma", ctypes.c_double),
        ("lam_min", ctypes.c_double),
        ("lam_max", ctypes.c_double),
        ("r_min", ctypes.c_double),
        ("r_max_frac", ctypes.c_double),
        ("p_two_mu", ctypes.c_double),
        ("p_one_mu", ctypes.c_double),
        ("slope_max", ctypes.c_double),
        ("sigma", ctypes.c_double),
    ]


@dataclass(frozen=True)
class Workload:
    """Shape of a synthetic workload.  ``window`` is the alignment window w in
    cm; the selection threshold it implies is chosen by the caller."""

    name: str
    seed: int
    n_events: int
    station_z: tuple
    bg_lambda: float = 20.0
    radial: str = "area"          # "area": uniform in area; "inv_r2": area density ~ 1/r^2
    lognormal: bool = False        # per-event lambda ~ log-normal (median, sigma_log), clipped
    ln_median: float = 60.0
    ln_sigma: float = 1.0
    count_min: int = 5
    count_max: int = 1500
    p_two_mu: float = 0.0
    p_one_mu: float = 0.0
    window: float = 0.5
    slope_max: float = 0.35
    sigma: float = 0.1
    r_min: float = 15.0
    r_max_frac: float = 0.4
    layer_dz: float = 10.0
    extra: dict = field(default_factory=dict, compare=False, hash=False)

    @property
    def n_stations(self) -> int:
        return len(self.station_z)


_Z4 = (130.0, 165.0, 200.0, 235.0)
_Z6 = (130.0, 165.0, 200.0, 235.0, 270.0, 305.0)

WORKLOADS = {
    # 1 000 events, Poisson(20) background per layer uniform in area, 30 % of
    # events with two muons.  Small enough for the oracle in seconds.
    "poisson20_1k": Workload("poisson20_1k", 1, 1000, _Z4, bg_lambda=20.0, radial="area", p_two_mu=0.30),
    # 10^6 events, Poisson(100) background per layer with 1/r^2 area density,
    # 1 % of events with two muons and 5 % with one.
    "poisson100_1m": Workload("poisson100_1m", 2, 1_000_000, _Z4, bg_lambda=100.0, radial="inv_r2",
                              p_two_mu=0.01, p_one_mu=0.05),
    # Uneven timeslices: per event lambda_e = clip(exp(ln 60 + N(0,1)), 5, 1500),
    # per layer count = clip(Poisson(lambda_e), 5, 1500); signal as above.
    # 64 timeslices of U[1e4, 1e5] events each (sizes from timeslice_sizes()).
    "lognormal_timeslices": Workload("lognormal_timeslices", 3, 0, _Z4, radial="inv_r2", lognormal=True,
                                     p_two_mu=0.01, p_one_mu=0.05,
                                     extra={"n_slices": 64, "slice_min": 10_000, "slice_max": 100_000}),
    # Streaming: timeslices of U[2e3, 2e5] events, Poisson arrivals at an
    # aggregate 1e7 events/s, multiplicities as above.
    "lognormal_stream": Workload("lognormal_stream", 4, 0, _Z4, radial="inv_r2", lognormal=True,
                                 p_two_mu=0.01, p_one_mu=0.05,
                                 extra={"slice_min": 2_000, "slice_max": 200_000, "rate_events_per_s": 1e7}),
    # Free-streaming timeslice: collisions of the poisson100_1m recipe (own
    # seed) at Poisson arrival times, 1e7 collisions/s (the interaction rate
    # CBM aims at, Sec. 1-2), every hit at its collision's time plus
    # N(0, 3 ns); windows of 100 ns, coincidence width 15 ns.  100 000
    # collisions (10 ms of beam) per timeslice.
    "poisson100_stream": Workload("poisson100_stream", 6, 100_000, _Z4, bg_lambda=100.0, radial="inv_r2",
                                  p_two_mu=0.01, p_one_mu=0.05,
                                  extra={"rate_hz": 1e7, "sigma_t_ns": 3.0, "window_ns": 100.0, "dt_ns": 15.0,
                                         "t0_ns": 100.0}),
    # Combinatorial stress: 6 stations, Poisson(1500) background per layer,
    # 10 % of events with two muons, window 1.0 cm.
    "poisson1500_6st": Workload("poisson1500_6st", 5, 200_000, _Z6, bg_lambda=1500.0, radial="inv_r2",
                                p_two_mu=0.10, window=1.0),
}


def build(force: bool = False) -> str:
    """Compile the generator (plain C, no FP contraction) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
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
        lib.jpsi_synth_counts.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_int]
        lib.jpsi_synth_fill.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int]
        lib.jpsi_synth_log.argtypes = [ctypes.c_double]
        lib.jpsi_synth_log.restype = ctypes.c_double
        lib.jpsi_synth_exp.argtypes = [ctypes.c_double]
        lib.jpsi_synth_exp.restype = ctypes.c_double
        lib.jpsi_synth_xoshiro_first.argtypes = [ctypes.c_uint64] * 4 + [ctypes.c_int, ctypes.c_void_p]
        lib.jpsi_synth_xoshiro_first.restype = ctypes.c_uint64
        lib.jpsi_synth_splitmix_mix.argtypes = [ctypes.c_uint64]
        lib.jpsi_synth_splitmix_mix.restype = ctypes.c_uint64
        _lib = lib
    return _lib


def _cfg(w: Workload) -> _Cfg:
    c = _Cfg()
    c.n_stations = w.n_stations
    c.radial = 1 if w.radial == "inv_r2" else 0
    c.bg_mode = 1 if w.lognormal else 0
    c.count_min, c.count_max = w.count_min, w.count_max
    for i, zc in enumerate(w.station_z):
        c.station_z[i] = zc
    c.layer_dz = w.layer_dz
    c.bg_lambda = w.bg_lambda
    c.ln_median, c.ln_sigma = w.ln_median, w.ln_sigma
    c.lam_min, c.lam_max = float(w.count_min), float(w.count_max)
    c.r_min, c.r_max_frac = w.r_min, w.r_max_frac
    c.p_two_mu, c.p_one_mu = w.p_two_mu, w.p_one_mu
    c.slope_max, c.sigma = w.slope_max, w.sigma
    return c


def default_threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def layer_counts(w: Workload, e0: int, n_events: int, n_threads: int | None = None, seed: int | None = None):
    """int32 [n_events, n_stations*3] hit counts per layer."""
    lib = _load()
    S3 = w.n_stations * 3
    counts = np.zeros((n_events, S3), dtype=np.int32)
    rc = lib.jpsi_synth_counts(ctypes.byref(_cfg(w)), w.seed if seed is None else seed, e0, n_events,
                               counts.ctypes.data, n_threads or default_threads())
    if rc:
        raise ValueError("jpsi_synth_counts rejected its arguments")
    return counts


def generate(w: Workload | str, e0: int = 0, n_events: int | None = None, *, n_threads: int | None = None,
             seed: int | None = None, truth: bool = False, out=None):
    """Events [e0, e0+n_events) of workload ``w``.

    Returns a dict with ``x, y, z`` (float32 [n_hits]), ``offsets`` (int32
    [n_events*S*3+1], batch-relative CSR over (event, station, layer)),
    ``n_events``, ``n_stations`` and optionally ``truth`` (int8 [n_hits]: 0
    background, 1/2 muon number).  ``out`` may supply preallocated x/y/z
    arrays (e.g. pinned host buffers viewed as numpy) of sufficient length.
    """
    if isinstance(w, str):
        w = WORKLOADS[w]
    if n_events is None:
        n_events = w.n_events
    lib = _load()
    nt = n_threads or default_threads()
    counts = layer_counts(w, e0, n_events, nt, seed)
    off64 = np.zeros(counts.size + 1, dtype=np.int64)
    np.cumsum(counts.reshape(-1), out=off64[1:])
    n_hits = int(off64[-1])
    if n_hits >= 2**31:
        raise ValueError(f"{n_hits} hits exceed int32 CSR offsets; generate fewer events per batch")
    if out is not None:
        x, y, z = out["x"][:n_hits], out["y"][:n_hits], out["z"][:n_hits]
    else:
        x = np.empty(n_hits, np.float32)
        y = np.empty(n_hits, np.float32)
        z = np.empty(n_hits, np.float32)
    tr = np.empty(n_hits, np.int8) if truth else None
    rc = lib.jpsi_synth_fill(ctypes.byref(_cfg(w)), w.seed if seed is None else seed, e0, n_events,
                             off64.ctypes.data, x.ctypes.data, y.ctypes.data, z.ctypes.data,
                             tr.ctypes.data if truth else None, nt)
    if rc:
        raise ValueError("jpsi_synth_fill rejected its arguments")
    res = {"x": x, "y": y, "z": z, "offsets": off64.astype(np.int32), "n_events": n_events,
           "n_stations": w.n_stations, "n_hits": n_hits, "workload": w.name}
    if truth:
        res["truth"] = tr
    return res


def timeslice_sizes(w: Workload | str, n_slices: int | None = None):
    """Event counts of the timeslices of a timeslice/stream workload (uniform
    in [slice_min, slice_max]); drawn with numpy's PCG64 from the workload seed."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    n = n_slices if n_slices is not None else w.extra.get("n_slices", 64)
    rng = np.random.Generator(np.random.PCG64(w.seed * 1_000_003 + 17))
    return rng.integers(w.extra["slice_min"], w.extra["slice_max"] + 1, size=n).astype(np.int64)


def arrival_times(w: Workload | str, sizes):
    """Poisson-process arrival times (s) of timeslices whose aggregate event
    rate is ``rate_events_per_s``: exponential gaps with mean = mean size / rate."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    rng = np.random.Generator(np.random.PCG64(w.seed * 1_000_003 + 29))
    mean_gap = float(np.mean(sizes)) / w.extra["rate_events_per_s"]
    return np.cumsum(rng.exponential(mean_gap, size=len(sizes)))


def timeslice(w: Workload | str, e0: int = 0, n_collisions: int | None = None, *, n_threads: int | None = None,
              rate_hz: float | None = None, sigma_t_ns: float | None = None, window_ns: float | None = None,
              dt_ns: float | None = None):
    """A free-streaming timeslice made of collisions [e0, e0+n) of workload
    ``w``'s event recipe.

    Collision c arrives at t0 + the sum of c+1 exponential gaps (mean
    1/rate); each of its hits is seen at that time plus N(0, sigma_t).  The
    hits of all collisions are merged per (station, layer) and each group is
    sorted by time (stably: ties keep collision, then hit order).  Times are
    float32 ns from the timeslice start (so their resolution is that of a
    float at the timeslice's length: 1 ns at 1e7 ns).  Windows are
    [k W, (k+1) W) up to past the last hit.  Returns x, y, z, t (float32
    [n_hits]), offsets (int32 [3S+1]), bounds (float32 [K+1]), dt,
    n_stations, n_hits, collision_times (float64 ns), batch_offsets (the
    generated events' offsets) and src (int64 [n_hits]: the index, in the
    generated batch, of each timeslice hit)."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    ex = w.extra
    n = w.n_events if n_collisions is None else n_collisions
    rate = rate_hz if rate_hz is not None else ex.get("rate_hz", 1e7)
    sig = sigma_t_ns if sigma_t_ns is not None else ex.get("sigma_t_ns", 3.0)
    W = window_ns if window_ns is not None else ex.get("window_ns", 100.0)
    dt = dt_ns if dt_ns is not None else ex.get("dt_ns", 15.0)
    b = generate(w, e0, n, n_threads=n_threads)
    S = w.n_stations
    S3 = 3 * S
    off = b["offsets"].astype(np.int64)
    counts = np.diff(off)                                  # [n * S3]: hits per (collision, group)
    rng = np.random.Generator(np.random.PCG64(w.seed * 1_000_003 + 41 + 7919 * e0))
    tc = ex.get("t0_ns", 100.0) + np.cumsum(rng.exponential(1e9 / rate, size=n))
    coll = np.repeat(np.repeat(np.arange(n), S3), counts)  # collision of each batch hit
    grp = np.repeat(np.tile(np.arange(S3), n), counts)     # layer group of each batch hit
    t_hit = (tc[coll] + rng.normal(0.0, sig, size=coll.size)).astype(np.float32)
    by_group = np.argsort(grp, kind="stable")              # batch hits grouped, batch order kept
    gsizes = np.bincount(grp, minlength=S3)
    goff = np.zeros(S3 + 1, np.int64)
    np.cumsum(gsizes, out=goff[1:])
    src = np.empty(coll.size, np.int64)
    for g in range(S3):
        idx = by_group[goff[g]:goff[g + 1]]
        src[goff[g]:goff[g + 1]] = idx[np.argsort(t_hit[idx], kind="stable")]
    t = t_hit[src]
    t_end = float(t.max()) if t.size else 0.0
    K = int(np.floor(max(t_end, 0.0) / W)) + 1
    bounds = (np.arange(K + 1, dtype=np.float64) * W).astype(np.float32)
    return {"x": b["x"][src], "y": b["y"][src], "z": b["z"][src], "t": t, "offsets": goff.astype(np.int32),
            "bounds": bounds, "dt": float(dt), "n_stations": S, "n_hits": int(src.size), "collision_times": tc,
            "src": src, "batch_offsets": b["offsets"], "n_collisions": n, "workload": w.name}


def checksum(batch) -> str:
    """Hash of the generated arrays (bytes), for determinism checks."""
    import hashlib
    h = hashlib.sha256()
    for k in ("offsets", "x", "y", "z"):
        h.update(np.ascontiguousarray(batch[k]).tobytes())
    return h.hexdigest()
