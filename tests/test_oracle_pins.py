"""Pins of the oracle against facts the paper and the mathematics fix.

The paper (Sec. 3.2) gives the method but no worked numeric example, so the
oracle is pinned by closed forms of the least-squares fit through the origin,
special cases (tracks from the target, zero window), invariances, brute force
and the paper's printed cut values and accept rule.
"""
from fractions import Fraction

import numpy as np
import pytest

from helpers import accept_list, line_event, make_batch, sorted_triplets

EPS = 2.0 ** -24


def exact_fit(u, z):
    """Least squares u = m z through the origin, in exact rationals:
    m* = sum(uz)/sum(z^2), S* = sum(u^2) - sum(uz)^2/sum(z^2)."""
    U = [Fraction(float(v)) for v in u]
    Z = [Fraction(float(v)) for v in z]
    szz = sum(a * a for a in Z)
    suz = sum(a * b for a, b in zip(U, Z))
    return suz / szz, sum(a * a for a in U) - suz * suz / szz


# ---------------------------------------------------------------- P1 closed forms

def test_closed_form_exact_line(oracle_mod):
    # z = (1,2,3), x = (1,2,3): x = 1*z exactly, S = 0 in any precision
    ok, mx, my, sx, sy = oracle_mod.triplet([1, 2, 3], [2, 4, 6], [1, 2, 3], 0.0, 0.0)
    assert (mx, my, sx, sy) == (1.0, 2.0, 0.0, 0.0)
    assert ok  # S = 0 <= C = 0: equality passes ("rejected if above", Sec. 3.2)


def test_closed_form_five_fourteenths(oracle_mod):
    # x = (1,2,4), z = (1,2,3): m* = 17/14, S* = 21 - 289/14 = 5/14
    m_star, s_star = exact_fit([1, 2, 4], [1, 2, 3])
    assert (m_star, s_star) == (Fraction(17, 14), Fraction(5, 14))
    ok, mx, _, sx, _ = oracle_mod.triplet([1, 2, 4], [0, 0, 0], [1, 2, 3], 1.0, 1.0)
    assert abs(Fraction(mx) - m_star) <= 4 * EPS * m_star
    assert abs(Fraction(sx) - s_star) <= 32 * EPS * Fraction(21)
    assert ok
    # cut just below / above 5/14 decides
    assert not oracle_mod.triplet([1, 2, 4], [0, 0, 0], [1, 2, 3], 0.357, 1.0)[0]
    assert oracle_mod.triplet([1, 2, 4], [0, 0, 0], [1, 2, 3], 0.3572, 1.0)[0]


def test_closed_form_random_rationals(oracle_mod):
    """FP32 S within a rounding bound of the exact S* = min_m sum (u - m z)^2;
    a dropped term, a wrong sign or a transposed operand breaks this."""
    rng = np.random.default_rng(11)
    for _ in range(400):
        z = np.sort(rng.uniform(50, 320, 3)).astype(np.float32)
        m = rng.uniform(-0.4, 0.4)
        u = (m * z.astype(np.float64) + rng.normal(0, rng.choice([0.01, 0.3, 3.0]), 3)).astype(np.float32)
        m_star, s_star = exact_fit(u, z)
        ok, mx, my, sx, sy = oracle_mod.triplet(list(u), list(u), list(z), 1e30, 1e30)
        assert mx == my and sx == sy
        scale = sum(Fraction(float(v)) ** 2 for v in u)
        assert abs(Fraction(mx) - m_star) <= 6 * EPS * abs(m_star) + Fraction(1, 10**30)
        # residual error: 2 |r| eps |m z| per hit plus relative rounding of the sums
        bound = 8 * EPS * (Fraction(float(np.sqrt(float(s_star)))) * Fraction(float(np.sqrt(float(scale)))) + s_star) \
            + 64 * EPS * EPS * scale
        assert abs(Fraction(sx) - s_star) <= bound


def test_pinned_order_matches_float32_stepwise(oracle_mod):
    """Cross-check of the evaluation order written out with numpy float32
    scalars (IEEE single, no contraction)."""
    rng = np.random.default_rng(5)
    f = np.float32
    for _ in range(2000):
        z = rng.uniform(100, 320, 3).astype(np.float32)
        x = (rng.uniform(-0.4, 0.4) * z + rng.normal(0, 0.5, 3)).astype(np.float32)
        szz = (f(z[0] * z[0]) + f(z[1] * z[1])) + f(z[2] * z[2])
        sxz = (f(x[0] * z[0]) + f(x[1] * z[1])) + f(x[2] * z[2])
        m = f(sxz / szz)
        r = [f(x[k] - f(m * z[k])) for k in range(3)]
        s = (f(r[0] * r[0]) + f(r[1] * r[1])) + f(r[2] * r[2])
        _, mx, _, sx, _ = oracle_mod.triplet(list(x), list(x), list(z), 0.5, 0.5)
        assert np.float32(mx) == m and np.float32(sx) == s


def test_paper_cut_values(oracle_mod):
    # Sec. 3.2 step 2b: MSD per dof thresholds 0.03 (xz) and 0.025 (yz); with
    # ndf = 2 the summed-square cut is exactly twice each float threshold
    c_xz, c_yz = oracle_mod.cut(2, 0.03), oracle_mod.cut(2, 0.025)
    assert c_xz == np.float32(0.03) * np.float32(2)
    assert c_yz == np.float32(0.025) * np.float32(2)
    # a residual with S in (0.05, 0.06): passes the xz cut, fails the yz cut,
    # so each plane is held to its own threshold
    z = [120.0, 130.0, 140.0]
    zero = [0.0, 0.0, 0.0]
    bump = [0.0, 0.287, 0.0]  # S* = 0.287^2 (1 - 130^2 / 50900) = 0.0550
    s = oracle_mod.triplet(zero, bump, z, 1.0, 1.0)[4]
    assert 0.05 < s < 0.06
    assert oracle_mod.triplet(bump, zero, z, c_xz, c_yz)[0]
    assert not oracle_mod.triplet(zero, bump, z, c_xz, c_yz)[0]


def test_nan_inf_never_pass(oracle_mod):
    z = [120.0, 130.0, 140.0]
    for bad in (np.nan, np.inf, -np.inf):
        for k in range(3):
            x = [0.0, 0.0, 0.0]
            x[k] = bad
            assert not oracle_mod.triplet(x, [0, 0, 0], z, 1e30, 1e30)[0]
            assert not oracle_mod.triplet([0, 0, 0], x, z, 1e30, 1e30)[0]
    for badz in (np.nan, np.inf):
        zz = list(z)
        zz[1] = badz
        assert not oracle_mod.triplet([1, 1, 1], [1, 1, 1], zz, 1e30, 1e30)[0]


# ------------------------------------------------------------ special cases

def test_tracks_from_target_always_found(oracle_mod):
    """Straight lines from the vertex (Sec. 3.1) pass for any cut >= 1e-6 cm^2,
    in every station, and chain into candidates."""
    rng = np.random.default_rng(3)
    events = []
    for _ in range(60):
        tracks = [tuple(rng.uniform(-0.35, 0.35, 2)) for _ in range(rng.integers(1, 4))]
        events.append(line_event(4, tracks, rng=rng, extra_bg=5))
    b = make_batch(events, 4)
    for t in (1e-6 / 2, 0.015, 0.25):
        r = oracle_mod.run(oracle_mod.params(4, oracle_mod.MODE_CHAIN, t_xz=t), b)
        n_tracks = [len(ev[0]) - 5 for ev in events]
        assert np.all(r["track_counts"] >= n_tracks)
        assert np.all(r["unit_counts"].reshape(-1, 4) >= np.array(n_tracks)[:, None])
        acc = accept_list(r["accept_bits"], len(events))
        assert np.all(acc[np.array(n_tracks) >= 2])


def test_zero_window_on_smeared_hits_gives_nothing(oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 200)
    for mode in (oracle_mod.MODE_PAPER, oracle_mod.MODE_CHAIN):
        r = oracle_mod.run(oracle_mod.params(4, mode, t_xz=0.0), b)
        assert r["trip_needed"] == 0 and not r["track_counts"].any() and not r["accept_bits"].any()


def test_empty_layers(oracle_mod):
    z = [120.0, 130.0, 140.0]
    ev = [[(0.0, 0.0, z[0])], [], [(0.0, 0.0, z[2])]]
    b = make_batch([ev], 1)
    for mode in (0, 1):
        r = oracle_mod.run(oracle_mod.params(1, mode, t_xz=1.0), b)
        assert r["status"] == 0 and r["trip_needed"] == 0 and r["track_counts"][0] == 0
    b = make_batch([], 4)
    r = oracle_mod.run(oracle_mod.params(4, 1), b)
    assert r["status"] == 0 and r["trip_needed"] == 0


def test_accept_needs_two_triplets(oracle_mod):
    """Sec. 3.2 step 3: at least two passing triplets (sharing hits allowed)."""
    z = [120.0, 130.0, 140.0]
    one = [[(0.12 * z[0], 0.0, z[0])], [(0.12 * z[1], 0.0, z[1])], [(0.12 * z[2], 0.0, z[2])]]
    # a second hit in the last layer close to the line: two triplets sharing two hits
    two = [one[0], one[1], one[2] + [(0.12 * z[2] + 0.01, 0.0, z[2])]]
    b = make_batch([one, two], 1)
    r = oracle_mod.run(oracle_mod.params(1, oracle_mod.MODE_PAPER, t_xz=0.03, t_yz=0.025), b)
    assert list(r["track_counts"]) == [1, 2]
    assert list(accept_list(r["accept_bits"], 2)) == [False, True]


def test_chain_single_station_equals_paper(oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 300)
    # view stations as independent one-station events (CSR over 1 station)
    b1 = dict(b, n_events=b["n_events"] * 4, n_stations=1)
    rp = oracle_mod.run(oracle_mod.params(1, oracle_mod.MODE_PAPER, t_xz=0.25), b1)
    rc = oracle_mod.run(oracle_mod.params(1, oracle_mod.MODE_CHAIN, t_xz=0.25), b1)
    assert np.array_equal(rp["track_counts"], rc["track_counts"])
    assert np.array_equal(rp["triplets"], rc["triplets"])


def test_chain_requires_every_station(oracle_mod):
    """A trigger triplet is a candidate only with a compatible passing triplet
    in each other station; a kink between stations or a missing station kills it."""
    rng = np.random.default_rng(9)
    straight = line_event(3, [(0.1, -0.2)], rng=rng)
    # station 0 replaced by another line from the target (slopes x1.05): it
    # passes on its own but is not compatible with the trigger triplet
    kinked = [list(l) for l in straight]
    for li in range(3):
        kinked[li] = [(x * 1.05, y * 1.05, z) for (x, y, z) in straight[li]]
    missing = [list(l) for l in straight]
    missing[4] = []  # station 1, middle layer: no triplet there
    b = make_batch([straight, kinked, missing], 3)
    r = oracle_mod.run(oracle_mod.params(3, oracle_mod.MODE_CHAIN, t_xz=0.25), b)
    assert list(r["track_counts"]) == [1, 0, 0]
    rp = oracle_mod.run(oracle_mod.params(3, oracle_mod.MODE_PAPER, t_xz=0.25), b)
    assert list(rp["track_counts"]) == [1, 1, 1]


# -------------------------------------------------------------- invariances

def _canon(r, n_units):
    return sorted_triplets(r["trip_off"], r["triplets"], n_units)


def test_mirror_and_swap_bit_exact(oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 300)
    n_units = 300 * 4
    base = oracle_mod.run(oracle_mod.params(4, 1, t_xz=0.25, t_yz=0.2), b)
    mir = oracle_mod.run(oracle_mod.params(4, 1, t_xz=0.25, t_yz=0.2), dict(b, x=-b["x"]))
    assert np.array_equal(_canon(base, n_units), _canon(mir, n_units))
    assert np.array_equal(base["track_counts"], mir["track_counts"])
    sw = oracle_mod.run(oracle_mod.params(4, 1, t_xz=0.2, t_yz=0.25), dict(b, x=b["y"], y=b["x"]))
    assert np.array_equal(_canon(base, n_units), _canon(sw, n_units))
    assert np.array_equal(base["track_counts"], sw["track_counts"])


def test_power_of_two_scaling_exact(oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 300)
    base = oracle_mod.run(oracle_mod.params(4, 1, t_xz=0.25), b)
    sc = oracle_mod.run(oracle_mod.params(4, 1, t_xz=1.0),
                        dict(b, x=b["x"] * 2, y=b["y"] * 2, z=b["z"] * 2))
    assert np.array_equal(base["triplets"], sc["triplets"])
    assert np.array_equal(base["track_counts"], sc["track_counts"])


def test_permutation_invariance(oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 200)
    rng = np.random.default_rng(4)
    off = b["offsets"].astype(np.int64)
    perm = np.arange(b["n_hits"])
    for l in range(len(off) - 1):
        seg = perm[off[l]:off[l + 1]]
        perm[off[l]:off[l + 1]] = seg[rng.permutation(len(seg))]
    bp = dict(b, x=b["x"][perm], y=b["y"][perm], z=b["z"][perm])
    p = oracle_mod.params(4, 1, t_xz=0.25)
    r0, r1 = oracle_mod.run(p, b), oracle_mod.run(p, bp)
    assert np.array_equal(r0["track_counts"], r1["track_counts"])
    assert np.array_equal(r0["unit_counts"], r1["unit_counts"])
    # map permuted layer-local indices back to the original ones
    local_orig = perm - np.repeat(off[:-1], np.diff(off))
    unit = np.repeat(np.arange(200 * 4), np.diff(r1["trip_off"]))
    t1 = r1["triplets"].astype(np.int64).copy()
    for c in range(3):
        layer = unit * 3 + c
        t1[:, c] = local_orig[off[layer] + t1[:, c]]
    a0 = _canon(r0, 800)
    a1 = sorted_triplets(r1["trip_off"], t1, 800)
    assert np.array_equal(a0, a1)


def test_monotone_in_cut(oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 200)
    prev = None
    for t in (0.0, 0.01, 0.05, 0.25, 1.0, 4.0):
        r = oracle_mod.run(oracle_mod.params(4, 0, t_xz=t), b)
        cur = {tuple(v) for v in _canon(r, 800)}
        if prev is not None:
            assert prev <= cur
        prev = cur


# --------------------------------------------------------- brute vs pruned

def _near_threshold_events(rng, n_events, n_per_layer, c):
    """Events whose triplets sit on the cut: tracks from the target with hit
    offsets chosen so S lands within a few ulps of C, plus background."""
    events = []
    for _ in range(n_events):
        ev = []
        z = [120.0, 130.0, 140.0]
        tx, ty = rng.uniform(-0.3, 0.3, 2)
        # residual pattern orthogonal to z, scaled so that S lands on C
        zv = np.array(z)
        v = np.array([1.0, -2.0, 1.0])
        v = v - (v @ zv) / (zv @ zv) * zv
        v = v / np.sqrt(v @ v) * np.sqrt(c) * rng.uniform(0.999, 1.001)
        for li in range(3):
            hits = [(tx * z[li] + v[li], ty * z[li] + v[li] * rng.uniform(0.99, 1.01), z[li])]
            for _ in range(n_per_layer):
                hits.append((rng.uniform(-50, 50), rng.uniform(-50, 50), z[li]))
            ev.append(hits)
        events.append(ev)
    return events


@pytest.mark.parametrize("mode", [0, 1])
def test_brute_equals_pruned_random(oracle_mod, synth_mod, mode):
    b = synth_mod.generate("poisson20_1k", 0, 150)
    for t in (0.0, 0.03, 0.25, 2.0):
        p = oracle_mod.params(4, mode, t_xz=t, t_yz=t * 0.8)
        r0, r1 = oracle_mod.run(p, b), oracle_mod.run(p, b, brute=True)
        assert np.array_equal(r0["triplets"], r1["triplets"])
        assert np.array_equal(r0["track_counts"], r1["track_counts"])


def test_brute_equals_pruned_adversarial(oracle_mod):
    rng = np.random.default_rng(12)
    for c in (0.5, 0.06, 1e-4):
        ev = _near_threshold_events(rng, 40, 6, c)
        b = make_batch(ev, 1)
        p = oracle_mod.params(1, 0, t_xz=c / 2, t_yz=c / 2)
        r0, r1 = oracle_mod.run(p, b), oracle_mod.run(p, b, brute=True)
        assert r0["trip_needed"] > 0
        assert np.array_equal(r0["triplets"], r1["triplets"])
    # extreme magnitudes: huge, tiny and subnormal coordinates, NaN/Inf
    odd = [np.float32(v) for v in (0.0, 1e-38, 1e-42, 3e38, -3e38, 1e20, -1e-20, np.nan, np.inf, 5.0, -5.0)]
    zodd = [np.float32(v) for v in (1e-42, 1e-20, 1.0, 130.0, 3e38, np.inf)]
    events = []
    for _ in range(30):
        ev = []
        for li in range(3):
            ev.append([(rng.choice(odd), rng.choice(odd), rng.choice(zodd)) for _ in range(5)])
        events.append(ev)
    b = make_batch(events, 1)
    for t in (0.0, 0.5, 1e30):
        p = oracle_mod.params(1, 1, t_xz=t)
        r0, r1 = oracle_mod.run(p, b), oracle_mod.run(p, b, brute=True)
        assert r0["status"] == 0
        assert np.array_equal(r0["triplets"], r1["triplets"])


def test_threads_do_not_change_results(oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 300)
    p = oracle_mod.params(4, 1, t_xz=0.25)
    r1, r4 = oracle_mod.run(p, b, n_threads=1), oracle_mod.run(p, b, n_threads=4)
    for k in ("triplets", "track_counts", "accept_bits", "trip_off"):
        assert np.array_equal(r1[k], r4[k])


# ------------------------------------------------------------------ errors

def test_invalid_inputs(oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 5)
    p = oracle_mod.params(4, 1)
    bad = dict(b, offsets=b["offsets"].copy())
    bad["offsets"][3] = bad["offsets"][4] + 1
    assert oracle_mod.run(p, bad)["status"] == oracle_mod.EINVAL
    bad = dict(b, offsets=b["offsets"].copy())
    bad["offsets"][-1] -= 1
    assert oracle_mod.run(p, bad)["status"] == oracle_mod.EINVAL
    zb = b["z"].copy()
    zb[7] = 0.0
    assert oracle_mod.run(p, dict(b, z=zb))["status"] == oracle_mod.EINVAL
    assert oracle_mod.run(oracle_mod.params(4, 1, trigger_station=4), b)["status"] == oracle_mod.EINVAL
    # capacity too small: counts valid, triplets not written
    r = oracle_mod.run(p, b)
    if r["trip_needed"] > 0:
        rc = oracle_mod.run(p, b, capacity=r["trip_needed"] - 1)
        assert rc["status"] == oracle_mod.ECAPACITY and rc["trip_needed"] == r["trip_needed"]
        assert np.array_equal(rc["track_counts"], r["track_counts"])


# --------------------------------------------------------------- FP64 audit

def test_fp64_audit_agrees_away_from_cut(oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 300)
    p = oracle_mod.params(4, 1, t_xz=0.25)
    r32, r64 = oracle_mod.run(p, b), oracle_mod.run(p, b, fp64=True)
    a = {tuple(v) for v in _canon(r32, 1200)}
    c = {tuple(v) for v in _canon(r64, 1200)}
    # flips are only possible within a relative 1e-5 of the cut; none expected here
    assert len(a ^ c) <= 2


def test_ndf_scales_the_cut(oracle_mod):
    # "MSD per dof <= t" is S <= fl32(ndf * t).  x = (1, 2, 4) at z = (1, 2, 3)
    # has S* = 5/14 = 0.357...: above 2 * 0.15 = 0.3, below 3 * 0.15 = 0.45
    assert oracle_mod.cut(3, 0.15) == np.float32(np.float32(3.0) * np.float32(0.15))
    ev = [[(1.0, 0.0, 1.0)], [(2.0, 0.0, 2.0)], [(4.0, 0.0, 3.0)]]
    b = make_batch([ev], 1)
    for ndf, passes in ((2, False), (3, True), (1, False)):
        r = oracle_mod.run(oracle_mod.params(1, 0, t_xz=0.15, ndf=ndf, min_candidates=1), b)
        assert r["status"] == 0 and int(r["unit_counts"][0]) == int(passes), ndf
        assert bool(accept_list(r["accept_bits"], 1)[0]) == passes


def test_min_candidates_threshold(oracle_mod):
    # exactly two passing triplets (two straight tracks, no other hits that
    # combine): accepted for min_candidates 0, 1, 2, rejected for 3; 0 accepts
    # an event without any triplet too
    z = [120.0, 130.0, 140.0]
    tracks = [(0.1, 0.2), (-0.25, 0.05)]
    ev = [[(tx * zz, ty * zz, zz) for tx, ty in tracks] for zz in z]
    empty = [[], [], []]
    b = make_batch([ev, empty], 1)
    for minc, acc in ((0, [True, True]), (1, [True, False]), (2, [True, False]), (3, [False, False])):
        r = oracle_mod.run(oracle_mod.params(1, 0, t_xz=0.01, min_candidates=minc), b)
        assert r["status"] == 0 and list(r["track_counts"]) == [2, 0]
        assert list(accept_list(r["accept_bits"], 2)) == acc, minc


def _shared_hit_event(with_third_track):
    """One station, t = 10 cm^2: two nearby tracks whose layer-0 and layer-2
    hits combine with the single layer-1 hit in all four ways, so every
    candidate uses that hit; optionally a third track far away."""
    z = [120.0, 130.0, 140.0]
    l0 = [(0.1 * z[0], 0.1 * z[0], z[0]), (0.1 * z[0] + 3.0, 0.1 * z[0], z[0])]
    l1 = [(0.1 * z[1] + 1.5, 0.1 * z[1], z[1])]
    l2 = [(0.1 * z[2], 0.1 * z[2], z[2]), (0.1 * z[2] + 3.0, 0.1 * z[2], z[2])]
    if with_third_track:
        for layer, zz in zip((l0, l1, l2), z):
            layer.append((-0.2 * zz, 0.15 * zz, zz))
    return [l0, l1, l2]


def test_distinct_hits_candidates_sharing_a_hit_count_as_one(oracle_mod):
    # Sec. 3.2 step 3, "at least two triplets", read with distinct_hits = 1:
    # two candidates that use the same hit are one track, not two
    b = make_batch([_shared_hit_event(False), _shared_hit_event(True)], 1)
    plain = oracle_mod.run(oracle_mod.params(1, 0, t_xz=10.0), b)
    dist = oracle_mod.run(oracle_mod.params(1, 0, t_xz=10.0, distinct_hits=1), b)
    assert plain["status"] == 0 and dist["status"] == 0
    assert list(plain["track_counts"]) == [4, 5] and list(dist["track_counts"]) == [4, 5]
    assert list(accept_list(plain["accept_bits"], 2)) == [True, True]
    assert list(accept_list(dist["accept_bits"], 2)) == [False, True]
    # min_candidates 0 and 1 read the same with and without the rule
    for minc, acc in ((0, [True, True]), (1, [True, True])):
        r = oracle_mod.run(oracle_mod.params(1, 0, t_xz=10.0, min_candidates=minc, distinct_hits=1), b)
        assert list(accept_list(r["accept_bits"], 2)) == acc
    # more than two pairwise disjoint candidates is not defined: refused
    r = oracle_mod.run(oracle_mod.params(1, 0, t_xz=10.0, min_candidates=3, distinct_hits=1), b)
    assert r["status"] == oracle_mod.EINVAL
