"""Pins of the free-streaming selection of the oracle (oracle.stream).

The paper's Outlook (Sec. 8) says that free-streaming data carry no event
association, so hit times and event building must enter the selection; it
gives no rule.  The rule pinned here (the oracle header states it): a
triplet counts only when its hits are coincident, max t <= fl32(min t + dt),
and it belongs to the window that holds its earliest time.  Pins: isolated
collisions in a stream select exactly like the same events built by hand;
one window at equal times is one event; a triplet across a window boundary
counts once; an independent Python restatement on tiny timeslices.
"""
import itertools

import numpy as np
import pytest

from helpers import accept_list, make_batch, sorted_triplets


def to_timeslice(events, S, times):
    """Hits of several events (lists of (x, y, z) per layer) with per-hit times
    `times[e][g]` into one timeslice grouped by (station, layer), each group
    sorted by time; returns the timeslice and, per event and group, the group
    index of each original hit."""
    groups = [[] for _ in range(3 * S)]
    for e, ev in enumerate(events):
        for g, layer in enumerate(ev):
            for q, (x, y, z) in enumerate(layer):
                groups[g].append((times[e][g][q], e, q, x, y, z))
    where = [[dict() for _ in range(3 * S)] for _ in events]
    xs, ys, zs, ts, off = [], [], [], [], [0]
    for g in range(3 * S):
        for pos, (t, e, q, x, y, z) in enumerate(sorted(groups[g], key=lambda r: (r[0], r[1], r[2]))):
            where[e][g][q] = pos
            xs.append(x)
            ys.append(y)
            zs.append(z)
            ts.append(t)
        off.append(len(xs))
    ts_ = {"x": np.array(xs, np.float32), "y": np.array(ys, np.float32), "z": np.array(zs, np.float32),
           "t": np.array(ts, np.float32), "offsets": np.array(off, np.int32)}
    return ts_, where


def events_of(batch, S):
    off = batch["offsets"]
    out = []
    for e in range(batch["n_events"]):
        ev = []
        for g in range(3 * S):
            a, b = off[e * 3 * S + g], off[e * 3 * S + g + 1]
            ev.append(list(zip(batch["x"][a:b].tolist(), batch["y"][a:b].tolist(), batch["z"][a:b].tolist())))
        out.append(ev)
    return out


@pytest.mark.parametrize("mode", [0, 1])
def test_isolated_collisions_select_like_events(oracle_mod, synth_mod, mode):
    # 150 collisions 1000 ns apart, each spread over 5 ns, dt = 10 ns, one
    # window per collision: window e must select exactly as event e
    S, n, W = 4, 150, 1000.0
    b = synth_mod.generate("poisson20_1k", 0, n)
    events = events_of(b, S)
    rng = np.random.default_rng(3)
    times = [[(e * W + 100.0 + rng.uniform(0, 5, len(layer))).astype(np.float32).tolist() for layer in ev]
             for e, ev in enumerate(events)]
    ts, where = to_timeslice(events, S, times)
    p = oracle_mod.params(S, mode, t_xz=0.25)
    ref = oracle_mod.run(p, b)
    got = oracle_mod.stream(p, ts, [e * W for e in range(n + 1)], 10.0)
    assert got["status"] == 0 and ref["trip_needed"] > 0
    for k in ("unit_counts", "track_counts", "trip_off", "accept_bits"):
        assert np.array_equal(got[k], ref[k]), k
    # the same rows, once event-local indices become timeslice group indices
    rows = sorted_triplets(ref["trip_off"], ref["triplets"], n * S)
    mapped = sorted((u, where[u // S][3 * (u % S)][i], where[u // S][3 * (u % S) + 1][j],
                     where[u // S][3 * (u % S) + 2][k]) for u, i, j, k in rows.tolist())
    assert [tuple(r) for r in sorted_triplets(got["trip_off"], got["triplets"], n * S).tolist()] == mapped


def test_one_window_at_equal_times_is_one_event(oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 7, 1)
    S = 4
    ts = {k: b[k] for k in ("x", "y", "z", "offsets")}
    ts["t"] = np.zeros(b["n_hits"], np.float32)
    for mode in (0, 1):
        p = oracle_mod.params(S, mode, t_xz=0.25)
        ref = oracle_mod.run(p, b)
        got = oracle_mod.stream(p, ts, [-1.0, 1.0], 0.0)
        for k in ("unit_counts", "track_counts", "trip_off", "accept_bits", "trip_needed"):
            assert np.array_equal(got[k], ref[k]), k
        assert np.array_equal(sorted_triplets(got["trip_off"], got["triplets"], S),
                              sorted_triplets(ref["trip_off"], ref["triplets"], S))


def test_triplet_across_a_window_boundary_counts_once(oracle_mod):
    # one straight track, hit times 9.0, 10.5, 11.0 ns, windows [0, 10), [10, 20)
    z = [120.0, 130.0, 140.0]
    ts = {"x": np.array([0.1 * v for v in z], np.float32), "y": np.array([0.05 * v for v in z], np.float32),
          "z": np.array(z, np.float32), "t": np.array([9.0, 10.5, 11.0], np.float32),
          "offsets": np.array([0, 1, 2, 3], np.int32)}
    p = oracle_mod.params(1, 0, t_xz=0.25, min_candidates=1)
    r = oracle_mod.stream(p, ts, [0.0, 10.0, 20.0], 3.0)
    assert list(r["unit_counts"]) == [1, 0] and list(accept_list(r["accept_bits"], 2)) == [True, False]
    # its hits span 2 ns: a 1.5 ns coincidence width drops it; exactly 2 keeps it
    assert oracle_mod.stream(p, ts, [0.0, 10.0, 20.0], 1.5)["trip_needed"] == 0
    assert oracle_mod.stream(p, ts, [0.0, 10.0, 20.0], 2.0)["trip_needed"] == 1
    # moved into the second window as a whole: counted there
    ts2 = dict(ts, t=ts["t"] + np.float32(4.0))
    assert list(oracle_mod.stream(p, ts2, [0.0, 10.0, 20.0], 3.0)["unit_counts"]) == [0, 1]


def test_invalid_timeslices(oracle_mod):
    z = [120.0, 130.0, 140.0]
    base = {"x": np.zeros(3, np.float32), "y": np.zeros(3, np.float32), "z": np.array(z, np.float32),
            "t": np.zeros(3, np.float32), "offsets": np.array([0, 1, 2, 3], np.int32)}
    p = oracle_mod.params(1, 0, t_xz=0.25)
    assert oracle_mod.stream(p, base, [0.0, 1.0], 0.0)["status"] == 0
    two = dict(base, x=np.zeros(4, np.float32), y=np.zeros(4, np.float32), z=np.array(z + [140.0], np.float32),
               t=np.array([0, 0, 5, 1], np.float32), offsets=np.array([0, 1, 2, 4], np.int32))
    assert oracle_mod.stream(p, two, [0.0, 10.0], 1.0)["status"] == oracle_mod.EINVAL  # a group out of time order
    nan = dict(base, t=np.array([0, np.nan, 0], np.float32))
    assert oracle_mod.stream(p, nan, [0.0, 1.0], 0.0)["status"] == oracle_mod.EINVAL
    assert oracle_mod.stream(p, base, [1.0, 1.0], 0.0)["status"] == oracle_mod.EINVAL  # empty window
    assert oracle_mod.stream(p, base, [0.0, 1.0], -1.0)["status"] == oracle_mod.EINVAL


def _restated(oracle_mod, ts, S, mode, t, bounds, dt, trig, minc=2):
    """The rule written out over Python lists (P1 and P2 from the oracle)."""
    f32 = np.float32
    off = ts["offsets"]
    cut = oracle_mod.cut(2, t)
    hit = lambda h: (float(ts["x"][h]), float(ts["y"][h]), float(ts["z"][h]))  # noqa: E731

    def coincident(times):
        return f32(max(times)) <= f32(f32(min(times)) + f32(dt))

    def passing(s):
        out = []
        groups = [range(off[3 * s + l], off[3 * s + l + 1]) for l in range(3)]
        for h0, h1, h2 in itertools.product(*groups):
            tt = [ts["t"][h0], ts["t"][h1], ts["t"][h2]]
            if not coincident(tt):
                continue
            a, b_, c = hit(h0), hit(h1), hit(h2)
            if oracle_mod.triplet([a[0], b_[0], c[0]], [a[1], b_[1], c[1]], [a[2], b_[2], c[2]], cut, cut)[0]:
                out.append(((h0 - off[3 * s], h1 - off[3 * s + 1], h2 - off[3 * s + 2]), (h0, h1, h2), min(tt)))
        return out

    def compatible(Th, th):  # P2 from an oracle micro-event run
        ev = [[hit(h)] for h in th] + [[hit(h)] for h in Th]
        r = oracle_mod.run(oracle_mod.params(2, 1, t_xz=t, min_candidates=1), make_batch([ev], 2))
        return int(r["track_counts"][0]) == 1

    allp = [passing(s) if (mode == 1 or s == trig) else [] for s in range(S)]
    K = len(bounds) - 1
    counts, tcounts, rows = [], [], []
    for k in range(K):
        own = lambda e: f32(bounds[k]) <= e[2] < f32(bounds[k + 1])  # noqa: E731
        per = [[e for e in allp[s] if own(e)] for s in range(S)]
        n_c = 0
        for T in per[trig]:
            if mode == 1 and S > 1:
                ok = all(any(coincident([ts["t"][h] for h in T[1] + u[1]]) and compatible(T[1], u[1])
                             for u in allp[s]) for s in range(S) if s != trig)
            else:
                ok = True
            n_c += ok
        tcounts.append(n_c)
        for s in range(S):
            counts.append(len(per[s]))
            rows += [(k * S + s,) + e[0] for e in per[s]]
    return counts, tcounts, sorted(rows)


@pytest.mark.parametrize("S,mode,trig", [(1, 0, 0), (2, 1, 1), (3, 1, 1), (3, 0, 2)])
def test_stream_restated(oracle_mod, S, mode, trig):
    rng = np.random.default_rng(50 + 10 * S + mode)
    # a few tracks at random times over 60 ns plus background; 6 windows of 10 ns
    events = [[[] for _ in range(3 * S)]]
    times = [[[] for _ in range(3 * S)]]
    for _ in range(6):
        tx, ty, t0 = rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(0, 60)
        for g in range(3 * S):
            zz = 120.0 + 35.0 * (g // 3) + 10.0 * (g % 3 - 1)
            if rng.random() < 0.9:
                events[0][g].append((tx * zz + rng.normal(0, 0.15), ty * zz + rng.normal(0, 0.15), zz))
                times[0][g].append(float(np.float32(t0 + rng.uniform(0, 2))))
    for g in range(3 * S):
        zz = 120.0 + 35.0 * (g // 3) + 10.0 * (g % 3 - 1)
        for _ in range(2):
            events[0][g].append((rng.uniform(-40, 40), rng.uniform(-40, 40), zz))
            times[0][g].append(float(np.float32(rng.uniform(0, 60))))
    ts, _ = to_timeslice(events, S, times)
    bounds = [0.0, 10.0, 20.0, 30.0, 40.0, 50.0, 60.0]
    for dt in (1.0, 3.0):
        counts, tcounts, rows = _restated(oracle_mod, ts, S, mode, 0.3, bounds, dt, trig)
        r = oracle_mod.stream(oracle_mod.params(S, mode, t_xz=0.3, trigger_station=trig), ts, bounds, dt)
        assert r["status"] == 0
        assert list(r["unit_counts"]) == counts
        assert list(r["track_counts"]) == tcounts
        assert list(accept_list(r["accept_bits"], len(bounds) - 1)) == [c >= 2 for c in tcounts]
        got = sorted(tuple(v) for v in sorted_triplets(r["trip_off"], r["triplets"], (len(bounds) - 1) * S).tolist())
        assert got == rows
    assert sum(counts) > 0


def _track(z, times, tx=0.1, ty=0.05):
    return {"x": np.array([tx * v for v in z], np.float32), "y": np.array([ty * v for v in z], np.float32),
            "z": np.array(z, np.float32), "t": np.array(times, np.float32),
            "offsets": np.arange(len(z) + 1, dtype=np.int32)}


def test_earliest_hit_on_a_boundary_belongs_to_the_later_window(oracle_mod):
    # windows are [b_k, b_k+1): a triplet whose earliest hit is exactly 10.0
    # belongs to [10, 20) only
    p = oracle_mod.params(1, 0, t_xz=0.25, min_candidates=1)
    r = oracle_mod.stream(p, _track([120.0, 130.0, 140.0], [10.0, 10.5, 11.0]), [0.0, 10.0, 20.0], 3.0)
    assert list(r["unit_counts"]) == [0, 1]


def test_latest_hit_on_the_rounded_range_end(oracle_mod):
    # a triplet owned by [0, 8) whose latest hit is exactly fl32(8 + dt): its
    # earliest time, the float just below 8, plus dt = 8.5 rounds up to 16.5
    # (the sum's ulp is four times the earliest time's)
    f32 = np.float32
    dt = f32(8.5)
    end = f32(f32(8.0) + dt)
    tau = np.nextafter(f32(8.0), f32(0.0))
    assert tau < f32(8.0) and f32(tau + dt) == end
    p = oracle_mod.params(1, 0, t_xz=0.25, min_candidates=1)
    r = oracle_mod.stream(p, _track([120.0, 130.0, 140.0], [tau, tau, end]), [0.0, 8.0, 16.0], float(dt))
    assert list(r["unit_counts"]) == [1, 0]


def test_chain_needs_the_stations_coincident(oracle_mod):
    # the same straight track in two stations: a candidate when both
    # stations' hits are within dt of each other, none when the upstream
    # station's hits come 30 ns later (each station alone is coincident)
    z = [120.0, 130.0, 140.0, 155.0, 165.0, 175.0]
    p = oracle_mod.params(2, 1, t_xz=0.25, min_candidates=1)
    for t_up, cand in ((1.0, 1), (30.0, 0)):
        ts = _track(z, [t_up, t_up, t_up, 1.0, 1.0, 1.0])
        r = oracle_mod.stream(p, ts, [0.0, 100.0], 5.0)
        assert r["status"] == 0 and list(r["unit_counts"]) == [1, 1] and list(r["track_counts"]) == [cand]


def test_chain_coincidence_at_the_last_ulp(oracle_mod):
    # trigger-station hits at 10 ns, dt = 4: the upstream station's hits chain
    # at 6 ns (max 10 <= fl32(6 + 4)) and not two ulps earlier
    # (fl32(6 - 2 ulp + 4) < 10)
    f32 = np.float32
    z = [120.0, 130.0, 140.0, 155.0, 165.0, 175.0]
    p = oracle_mod.params(2, 1, t_xz=0.25, min_candidates=1)
    early = np.nextafter(np.nextafter(f32(6.0), f32(0.0)), f32(0.0))
    assert f32(early + f32(4.0)) < f32(10.0)
    for t_up, cand in ((f32(6.0), 1), (early, 0)):
        ts = _track(z, [t_up, t_up, t_up, 10.0, 10.0, 10.0])
        r = oracle_mod.stream(p, ts, [0.0, 100.0], 4.0)
        assert r["status"] == 0 and list(r["track_counts"]) == [cand], t_up
