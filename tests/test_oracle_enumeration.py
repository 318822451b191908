"""An independent restatement of the oracle's loops, on tiny events.

The brute-force mode of the oracle shares its event and station loops with
the pruned mode, so brute == pruned pins the pair early-out but not the
enumeration itself.  Here every triple of every station is listed with
itertools.product over the per-layer hit lists, in Python, and decided by
the oracle's single-triplet predicate alone (P1 of Sec. 3.2, step 2).  The
CHAIN compatibility of a station triplet t with a trigger triplet T (no
refit) is taken from oracle runs on micro-events that hold exactly t's and
T's hits, one per layer, where no enumeration is left to get wrong.  From
these the test rebuilds the passing triplets of every unit, the candidates,
the track counts, the accept bits (step 3: at least min_candidates) and the
offsets, and compares them with oracle.run.
"""
import itertools

import numpy as np
import pytest

from helpers import accept_list, make_batch, sorted_triplets


def _tiny_events(rng, n_events, S, max_hits=4):
    """Events of 0..max_hits hits per layer: a few straight tracks from the
    target with small smear (so triplets pass and chain) plus background,
    shuffled; some layers empty."""
    zs = [120.0 + 35.0 * s + 10.0 * (l - 1) for s in range(S) for l in range(3)]
    events = []
    for _ in range(n_events):
        tracks = [tuple(rng.uniform(-0.3, 0.3, 2)) for _ in range(rng.integers(0, 4))]
        ev = []
        for z in zs:
            hits = []
            for tx, ty in tracks:
                if rng.random() < 0.95:
                    hits.append((tx * z + rng.normal(0, 0.15), ty * z + rng.normal(0, 0.15), z))
            while len(hits) < max_hits and rng.random() < 0.5:
                hits.append((rng.uniform(-40, 40), rng.uniform(-40, 40), z))
            rng.shuffle(hits)
            ev.append(hits[:max_hits])
        events.append(ev)
    return events


def _shared_hit_event(S, third):
    """Every station: two close tracks in layers 0 and 2 and one middle-layer
    hit between them, so the trigger station's candidates all use that hit;
    `third` adds a separate track."""
    ev = []
    for s in range(S):
        for l in range(3):
            z = 120.0 + 35.0 * s + 10.0 * (l - 1)
            hits = [(0.1 * z + 0.4, 0.1 * z, z)] if l == 1 else [(0.1 * z, 0.1 * z, z), (0.1 * z + 0.8, 0.1 * z, z)]
            if third:
                hits.append((-0.2 * z, 0.15 * z, z))
            ev.append(hits)
    return ev


class Restated:
    """Sec. 3.2 steps 1-3 (plus the CHAIN rule) over Python lists."""

    def __init__(self, oracle_mod, S, mode, t, ndf, minc, trig):
        self.o = oracle_mod
        self.S, self.mode, self.t, self.ndf, self.minc, self.trig = S, mode, t, ndf, minc, trig
        self.cut = oracle_mod.cut(ndf, t)
        self._compat = {}

    def passing(self, station):
        """Every (i, j, k) of the station's layers that passes P1, with its hits."""
        out = []
        for (i, a), (j, b), (k, c) in itertools.product(*(list(enumerate(layer)) for layer in station)):
            xs, ys, zs = [a[0], b[0], c[0]], [a[1], b[1], c[1]], [a[2], b[2], c[2]]
            if self.o.triplet(xs, ys, zs, self.cut, self.cut)[0]:
                out.append(((i, j, k), (a, b, c)))
        return out

    def compatible(self, T_hits, t_hits):
        """P2 from the oracle on a two-station micro-event: station 0 holds
        t's hits, the trigger station 1 holds T's; one candidate iff t is
        compatible with T (both pass P1)."""
        key = (T_hits, t_hits)
        if key not in self._compat:
            ev = [[h] for h in t_hits] + [[h] for h in T_hits]
            b = make_batch([ev], 2)
            r = self.o.run(self.o.params(2, 1, t_xz=self.t, t_yz=self.t, ndf=self.ndf, min_candidates=1), b)
            assert r["status"] == 0 and r["unit_counts"][0] == 1 and r["unit_counts"][1] == 1
            self._compat[key] = int(r["track_counts"][0]) == 1
        return self._compat[key]

    def event(self, ev):
        """Passing triplets per station, the candidates' (i, j, k), and whether
        two candidates share no hit."""
        stations = [ev[3 * s: 3 * s + 3] for s in range(self.S)]
        per = [self.passing(st) if (self.mode == 1 or s == self.trig) else [] for s, st in enumerate(stations)]
        T = per[self.trig]
        if self.mode == 0 or self.S == 1:
            cands = [ijk for ijk, _ in T]
        else:
            cands = [ijk for ijk, Th in T
                     if all(any(self.compatible(Th, th) for _, th in per[s]) for s in range(self.S) if s != self.trig)]
        disjoint = any(all(a != b for a, b in zip(c1, c2)) for c1, c2 in itertools.combinations(cands, 2))
        return per, len(cands), disjoint


@pytest.mark.parametrize("S,mode,trig", [(2, 1, 1), (3, 1, 2), (4, 1, 1), (3, 0, 2), (1, 1, 0)])
@pytest.mark.parametrize("ndf,minc,distinct", [(2, 2, 0), (3, 1, 0), (2, 3, 0), (2, 2, 1), (3, 1, 1)])
def test_enumeration_restated(oracle_mod, S, mode, trig, ndf, minc, distinct):
    rng = np.random.default_rng(1000 * S + 10 * mode + trig + 7 * ndf + minc)
    t = 0.3
    events = _tiny_events(rng, 40, S) + [_shared_hit_event(S, False), _shared_hit_event(S, True)]
    b = make_batch(events, S)
    R = Restated(oracle_mod, S, mode, t, ndf, minc, trig)
    counts, tcounts, rows, accepts = [], [], [], []
    for e, ev in enumerate(events):
        per, n_cand, disjoint = R.event(ev)
        tcounts.append(n_cand)
        accepts.append(disjoint if (distinct and minc == 2) else n_cand >= minc)
        for s in range(S):
            counts.append(len(per[s]))
            rows += [(e * S + s,) + ijk for ijk, _ in per[s]]
    # the events exercise chaining and both sides of the accept rule
    assert min(tcounts) < minc <= max(tcounts), (min(tcounts), max(tcounts))
    if distinct and minc == 2:  # some event needs the rule: two candidates, every pair sharing a hit
        assert any(c >= 2 and not a for c, a in zip(tcounts, accepts)), tcounts
    for brute in (False, True):
        r = oracle_mod.run(oracle_mod.params(S, mode, t_xz=t, ndf=ndf, min_candidates=minc, trigger_station=trig,
                                             distinct_hits=distinct), b, brute=brute)
        assert r["status"] == 0
        assert list(r["unit_counts"]) == counts
        assert list(r["track_counts"]) == tcounts
        assert list(r["trip_off"]) == [0] + list(np.cumsum(counts))
        assert list(accept_list(r["accept_bits"], len(events))) == accepts
        got = sorted_triplets(r["trip_off"], r["triplets"], len(events) * S)
        assert [tuple(v) for v in got] == sorted(rows)
