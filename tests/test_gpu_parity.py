"""GPU library (through the C ABI) == oracle, bit-exact, on seeded inputs of
every workload shape, plus the edge cases and error paths of the contract."""
import numpy as np
import pytest

from gpu_helpers import assert_same, gpu_select
from helpers import layer_z, line_event, make_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1810_11966_gb300 as jp
    jp.load(build_if_missing=True)
    return jp


def _ctx(lib, S=4, mode=1, t_xz=0.25, t_yz=None, **kw):
    return lib.Context(lib.params(S, mode, t_xz=t_xz, t_yz=t_yz), **kw)


def _oracle(oracle_mod, S, mode, t_xz, t_yz, batch, threads=8):
    return oracle_mod.run(oracle_mod.params(S, mode, t_xz=t_xz, t_yz=t_yz), batch, n_threads=threads)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("cuts", [(0.25, 0.25), (0.03, 0.025)])
@pytest.mark.parametrize("form", ["plain", "batched"])
def test_small_workload(lib, oracle_mod, synth_mod, mode, cuts, form):
    b = synth_mod.generate("poisson20_1k")
    ref = _oracle(oracle_mod, 4, mode, *cuts, b)
    ctx = _ctx(lib, 4, mode, *cuts)
    g = gpu_select(ctx, b, form=form)
    assert_same(g, ref, 4000, label=f"mode{mode} {cuts} {form}")


@pytest.mark.parametrize("mode", [0, 1])
def test_poisson100_slice(lib, oracle_mod, synth_mod, mode):
    # 3 000 events of the 10^6-event workload: several warp tiles, full bins
    b = synth_mod.generate("poisson100_1m", 0, 3000)
    ref = _oracle(oracle_mod, 4, mode, 0.25, 0.25, b)
    ctx = _ctx(lib, 4, mode)
    for form in ("plain", "batched"):
        assert_same(gpu_select(ctx, b, form=form), ref, 12000, label=form)


def test_lognormal_timeslice(lib, oracle_mod, synth_mod):
    # log-normal multiplicities: light events on warps, heavy ones on blocks
    b = synth_mod.generate("lognormal_timeslices", 0, 2500)
    counts = np.diff(b["offsets"]).reshape(-1, 12)
    assert counts.max() > 256  # exercises the block-per-event path
    ref = _oracle(oracle_mod, 4, 1, 0.25, 0.25, b)
    ctx = _ctx(lib, 4, 1)
    for form in ("plain", "batched"):
        assert_same(gpu_select(ctx, b, form=form), ref, 10000, label=form)


def test_stress_subset(lib, oracle_mod, synth_mod):
    # 6 stations x 1500 hits per layer, window 1.0 cm: ~10^4 triplets per unit
    b = synth_mod.generate("poisson1500_6st", 0, 60)
    ref = _oracle(oracle_mod, 6, 1, 1.0, 1.0, b, threads=16)
    assert ref["trip_needed"] > 60 * 6 * 1000
    ctx = _ctx(lib, 6, 1, 1.0)
    assert_same(gpu_select(ctx, b), ref, 360)


def test_adversarial_events(lib, oracle_mod):
    rng = np.random.default_rng(21)
    events = []
    # near-threshold straight tracks + background
    for _ in range(60):
        tracks = [tuple(rng.uniform(-0.35, 0.35, 2)) for _ in range(3)]
        events.append(line_event(2, tracks, rng=rng, sigma=0.3, extra_bg=8))
    # odd magnitudes, NaN, Inf, subnormal and huge z (z > 0 everywhere)
    odd = np.array([0.0, 1e-38, 1e-42, 3e38, -3e38, 1e20, -1e-20, np.nan, np.inf, -np.inf, 5.0, -5.0],
                   np.float32)
    zodd = np.array([1e-42, 1e-20, 1.0, 130.0, 3e38, np.inf, np.nan], np.float32)
    for _ in range(40):
        ev = []
        for _l in range(6):
            ev.append([(rng.choice(odd), rng.choice(odd), rng.choice(zodd)) for _ in range(rng.integers(0, 5))])
        events.append(ev)
    # empty event, one-hit event, empty middle layer
    events.append([[] for _ in range(6)])
    events.append([[(1.0, 1.0, 120.0)]] + [[] for _ in range(5)])
    zl = [120.0, 130.0, 140.0, 155.0, 165.0, 175.0]
    events.append([[(0.1 * z, 0.1 * z, z)] if li != 4 else [] for li, z in enumerate(zl)])
    b = make_batch(events, 2)
    for t in (0.0, 0.25, 1e30):
        for mode in (0, 1):
            ref = _oracle(oracle_mod, 2, mode, t, t, b)
            assert ref["status"] == 0
            ctx = _ctx(lib, 2, mode, t, t)
            for form in ("plain", "batched"):
                assert_same(gpu_select(ctx, b, form=form), ref, len(events) * 2, label=f"t={t} mode={mode} {form}")


def test_one_station_and_trigger_choice(lib, oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 400)
    b1 = dict(b, n_events=b["n_events"] * 4, n_stations=1)
    for mode in (0, 1):
        ref = _oracle(oracle_mod, 1, mode, 0.25, 0.25, b1)
        assert_same(gpu_select(_ctx(lib, 1, mode), b1), ref, 1600)
    # trigger station in the middle
    ref = oracle_mod.run(oracle_mod.params(4, 1, t_xz=0.25, trigger_station=1), b, n_threads=8)
    ctx = lib.Context(lib.params(4, 1, t_xz=0.25, trigger_station=1))
    assert_same(gpu_select(ctx, b), ref, 1600)


def test_zero_events(lib):
    ctx = _ctx(lib)
    b = make_batch([], 4)
    g = gpu_select(ctx, b)
    assert g["status"] == 0 and g["trip_needed"] == 0 and g["trip_off"][0] == 0


def test_many_tiny_events_ragged(lib, oracle_mod):
    # 70 001 events (not a multiple of any block), most with empty layers
    rng = np.random.default_rng(8)
    n = 70001
    counts = rng.integers(0, 3, size=(n, 6)).astype(np.int32)
    counts[rng.random(n) < 0.5] = 0
    off = np.zeros(counts.size + 1, np.int64)
    np.cumsum(counts.reshape(-1), out=off[1:])
    nh = int(off[-1])
    z = np.repeat(np.tile(np.array([120, 130, 140, 155, 165, 175], np.float32), n), counts.reshape(-1))
    t = rng.uniform(-0.1, 0.1, nh).astype(np.float32)
    b = {"x": (t * z + rng.normal(0, 0.2, nh)).astype(np.float32),
         "y": (t * z + rng.normal(0, 0.2, nh)).astype(np.float32),
         "z": z, "offsets": off.astype(np.int32), "n_events": n, "n_hits": nh}
    ref = _oracle(oracle_mod, 2, 1, 0.25, 0.25, b)
    assert_same(gpu_select(_ctx(lib, 2, 1), b), ref, 2 * n)


def test_invalid_inputs(lib, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 50)
    ctx = _ctx(lib)
    bad = dict(b, offsets=b["offsets"].copy())
    bad["offsets"][30] = bad["offsets"][31] + 5
    assert gpu_select(ctx, bad, triplets=False)["status"] == lib.JPSI_EINVAL
    bad = dict(b, offsets=b["offsets"].copy())
    bad["offsets"][-1] -= 1
    assert gpu_select(ctx, dict(bad, n_hits=b["n_hits"]), triplets=False)["status"] == lib.JPSI_EINVAL
    zb = b["z"].copy()
    zb[100] = -1.0
    assert gpu_select(ctx, dict(b, z=zb), triplets=False)["status"] == lib.JPSI_EINVAL
    # the context stays usable after an error
    assert gpu_select(ctx, b)["status"] == 0


def test_host_pointer_rejected(lib, synth_mod):
    import ctypes
    ctx = _ctx(lib)
    b = synth_mod.generate("poisson20_1k", 0, 10)
    hb = lib.make_batch(b["x"], b["y"], b["z"], b["offsets"], 10)
    o = lib.jpsi_outputs()
    import torch
    tc = torch.empty(10, dtype=torch.int32, device="cuda")
    o.track_counts = tc.data_ptr()
    s = lib.jpsi_run(ctx.ctx, hb, o, torch.cuda.current_stream().cuda_stream)
    # pageable host memory is only accepted where the device can address it
    if s != lib.JPSI_OK:
        assert s == lib.JPSI_EINVAL


def test_capacity_and_retry(lib, oracle_mod, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 300)
    ref = _oracle(oracle_mod, 4, 1, 0.25, 0.25, b)
    ctx = _ctx(lib)
    g = gpu_select(ctx, b, capacity=ref["trip_needed"] - 1)
    assert g["status"] == lib.JPSI_ECAPACITY and g["trip_needed"] == ref["trip_needed"]
    assert np.array_equal(g["track_counts"], ref["track_counts"])
    assert np.array_equal(g["trip_off"], ref["trip_off"])
    g = gpu_select(ctx, b, capacity=g["trip_needed"])
    assert_same(g, ref, 1200)


def test_budget_enomem(lib, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 1000)
    ctx = _ctx(lib, hbm_budget=4096)
    g = gpu_select(ctx, b, triplets=False)
    assert g["status"] == lib.JPSI_ENOMEM


def test_plain_equals_batched_and_deterministic(lib, synth_mod):
    b = synth_mod.generate("poisson100_1m", 5000, 20000)
    ctx = _ctx(lib)
    a = gpu_select(ctx, b, form="plain")
    for _ in range(2):
        c = gpu_select(ctx, b, form="batched")
        assert_same(c, a, 80000)


def test_run_host_matches_device(lib, synth_mod):
    import ctypes
    b = synth_mod.generate("poisson20_1k", 0, 700)
    ctx = _ctx(lib)
    dev = gpu_select(ctx, b)
    n = 700
    acc = np.zeros((n + 31) // 32, np.uint32)
    tc = np.zeros(n, np.int32)
    to = np.zeros(n * 4 + 1, np.int64)
    tr = np.zeros((dev["trip_needed"] + 5, 3), np.int32)
    o = lib.jpsi_outputs()
    o.accept_bits, o.track_counts, o.trip_off, o.triplets = acc.ctypes.data, tc.ctypes.data, to.ctypes.data, tr.ctypes.data
    o.trip_capacity = len(tr)
    hb = lib.make_batch(b["x"], b["y"], b["z"], b["offsets"], n)
    s = lib.jpsi_run_host(ctx.ctx, hb, o, 0)
    assert s == 0 and o.trip_needed == dev["trip_needed"]
    host = {"status": 0, "trip_needed": o.trip_needed, "accept_bits": acc, "track_counts": tc, "trip_off": to,
            "triplets": tr[: o.trip_needed]}
    assert_same(host, dev, n * 4)


def test_autotune_keeps_results(lib, synth_mod):
    import torch
    b = synth_mod.generate("lognormal_timeslices", 0, 4000)
    ctx = _ctx(lib)
    before = gpu_select(ctx, b)
    d = {k: torch.from_numpy(b[k]).cuda() for k in ("x", "y", "z", "offsets")}
    s = lib.jpsi_autotune(ctx.ctx, lib.make_batch(d["x"], d["y"], d["z"], d["offsets"], 4000))
    assert s == 0
    after = gpu_select(ctx, b)
    assert_same(after, before, 16000)


def test_dense_trigger_moves_to_block_tile(lib, oracle_mod):
    # 9 hits per layer on nearly one line: 9^3 passing trigger triplets, more
    # than a warp keeps, so the event runs on the block tile
    rng = np.random.default_rng(31)
    events = []
    for _ in range(20):
        tx, ty = rng.uniform(-0.3, 0.3, 2)
        zl = [120.0, 130.0, 140.0, 155.0, 165.0, 175.0]
        ev = []
        for z in zl:
            ev.append([(tx * z + rng.normal(0, 0.05), ty * z + rng.normal(0, 0.05), z) for _ in range(9)])
        events.append(ev)
    b = make_batch(events, 2)
    for mode in (0, 1):
        ref = _oracle(oracle_mod, 2, mode, 0.25, 0.25, b)
        assert ref["track_counts"].max() > 64
        ctx = _ctx(lib, 2, mode)
        for form in ("plain", "batched"):
            assert_same(gpu_select(ctx, b, form=form), ref, 40, label=f"mode={mode} {form}")


def _edge_residuals(z, C, pair, frac):
    """Residuals of a triplet at the edge of the pair pruning bound: the fit's
    residual vector r (orthogonal to z, so the least-squares slope is exactly
    the one the hits were placed on) along e_a/z_a - e_b/z_b, the direction
    that puts hits a and b furthest apart in slope for a given S = |r|^2 =
    frac * C."""
    z = np.asarray(z, float)
    v = np.zeros(3)
    v[pair[0]], v[pair[1]] = 1.0 / z[pair[0]], -1.0 / z[pair[1]]
    r = v - (v @ z) / (z @ z) * z
    return r * np.sqrt(frac * C / (r @ r))


@pytest.mark.parametrize("t", [0.25, 9e-4, 4.0])
def test_pair_bound_edge(lib, oracle_mod, t):
    # Triplets whose two hits sit as far apart in slope as a passing fit
    # allows (S just below, at and just above the cut), for every layer pair,
    # in both planes, among 10, 250 and 700 background hits per layer (small,
    # medium and block tiles): the pair pruning must keep every passing one.
    rng = np.random.default_rng(41)
    C = float(np.float32(2.0 * np.float32(t)))
    zl = layer_z(2)
    pairs = ((0, 1), (0, 2), (1, 2))
    events = []
    for n_bg in (10, 250, 700):
        for _ in range(4):
            ev = [[] for _ in range(6)]
            for s in range(2):
                z = zl[3 * s:3 * s + 3]
                for px in pairs:
                    for frac in (1.0 - 1e-3, 1.0 - 1e-6, 1.0, 1.0 + 1e-6):
                        py = pairs[rng.integers(3)]
                        mx, my = rng.uniform(-0.3, 0.3, 2)
                        rx, ry = _edge_residuals(z, C, px, frac), _edge_residuals(z, C, py, frac)
                        for li in range(3):
                            ev[3 * s + li].append((mx * z[li] + rx[li], my * z[li] + ry[li], z[li]))
                for li in range(3):
                    rr = rng.uniform(15.0, 0.4 * z[li], n_bg)
                    ph = rng.uniform(0, 2 * np.pi, n_bg)
                    ev[3 * s + li] += [(float(a * np.cos(q)), float(a * np.sin(q)), z[li]) for a, q in zip(rr, ph)]
                    rng.shuffle(ev[3 * s + li])
            events.append(ev)
    b = make_batch(events, 2)
    for mode in (0, 1):
        ref = _oracle(oracle_mod, 2, mode, t, t, b)
        assert ref["status"] == 0
        if mode == 1:  # the three triplets 1e-3 below the cut pass in every unit
            assert (ref["unit_counts"] >= 3).all()
        ctx = _ctx(lib, 2, mode, t, t)
        for form in ("plain", "batched"):
            assert_same(gpu_select(ctx, b, form=form), ref, len(events) * 2, label=f"t={t} mode={mode} {form}")


def test_huge_layer_goes_unpruned(lib, oracle_mod):
    # a layer above the block tile's 2048 hits: the unpruned kernel takes it
    rng = np.random.default_rng(32)
    events = []
    for n in (2100, 50, 2300):
        z = [120.0, 130.0, 140.0]
        ev = []
        for li in range(3):
            m = n if li == 1 else 40
            r = rng.uniform(15, 0.4 * z[li], m)
            ph = rng.uniform(0, 2 * np.pi, m)
            hits = [(float(a * np.cos(p)), float(a * np.sin(p)), z[li]) for a, p in zip(r, ph)]
            hits.append((0.1 * z[li], -0.05 * z[li], z[li]))
            ev.append(hits)
        events.append(ev)
    b = make_batch(events, 1)
    ref = _oracle(oracle_mod, 1, 1, 0.25, 0.25, b)
    assert ref["trip_needed"] >= 3
    assert_same(gpu_select(_ctx(lib, 1, 1), b), ref, 3)


def test_run_host_pipelined_matches_device(lib, synth_mod):
    # large enough that jpsi_run_host copies and counts in overlapping chunks
    n = 300_001
    b = synth_mod.generate("poisson20_1k", 0, n)
    ctx = _ctx(lib)
    dev = gpu_select(ctx, b)
    acc = np.zeros((n + 31) // 32, np.uint32)
    tc = np.zeros(n, np.int32)
    to = np.zeros(n * 4 + 1, np.int64)
    tr = np.zeros((dev["trip_needed"] + 1, 3), np.int32)
    o = lib.jpsi_outputs()
    o.accept_bits, o.track_counts, o.trip_off, o.triplets = acc.ctypes.data, tc.ctypes.data, to.ctypes.data, tr.ctypes.data
    o.trip_capacity = len(tr)
    hb = lib.make_batch(b["x"], b["y"], b["z"], b["offsets"], n)
    for _ in range(2):
        s = lib.jpsi_run_host(ctx.ctx, hb, o, 0)
        assert s == 0 and o.trip_needed == dev["trip_needed"]
        host = {"status": 0, "trip_needed": o.trip_needed, "accept_bits": acc, "track_counts": tc, "trip_off": to,
                "triplets": tr[: o.trip_needed]}
        assert_same(host, dev, n * 4)
    # too small a capacity: counts complete, ECAPACITY
    o.trip_capacity = dev["trip_needed"] - 1
    assert lib.jpsi_run_host(ctx.ctx, hb, o, 0) == lib.JPSI_ECAPACITY
    assert o.trip_needed == dev["trip_needed"] and np.array_equal(tc, dev["track_counts"])


def _block_tile_events(rng, n_events, S, odd_hit=None):
    """Events of about 500 hits in the middle layer of every station (past
    the warp tiles), each with a few hits along one line from the target."""
    zs = [130.0 + 35.0 * s + 10.0 * (li - 1) for s in range(S) for li in range(3)]
    events = []
    for k in range(n_events):
        tx, ty = rng.uniform(-0.3, 0.3, 2)
        ev = []
        for q, z in enumerate(zs):
            m = 500 if q % 3 == 1 else 60
            r = rng.uniform(15, 0.4 * z, m)
            ph = rng.uniform(0, 2 * np.pi, m)
            hits = [(float(a * np.cos(p)), float(a * np.sin(p)), z) for a, p in zip(r, ph)]
            hits += [(tx * z + rng.normal(0, 0.05), ty * z + rng.normal(0, 0.05), z) for _ in range(3)]
            if odd_hit is not None and k % 3 == 0 and q == 2:  # station 0, a non-trigger station
                hits.insert(int(rng.integers(len(hits))), odd_hit)
            ev.append(hits)
        events.append(ev)
    return make_batch(events, S)


def test_block_tile_station_blocks_hand_events_on(lib, oracle_mod):
    # CHAIN on block-tile events: the stations other than the trigger run on
    # their own blocks.  In every third event station 0 holds a finite hit
    # whose slope overflows (x = 3e38 at z = 0.1), so the block of that
    # station hands the event to the unpruned kernel; the rest stay split.
    rng = np.random.default_rng(41)
    b = _block_tile_events(rng, 12, 3, odd_hit=(3.0e38, 1.0, 0.1))
    ref = _oracle(oracle_mod, 3, 1, 0.25, 0.25, b)
    assert ref["track_counts"].max() > 0
    ctx = _ctx(lib, 3, 1)
    for form in ("plain", "batched"):
        assert_same(gpu_select(ctx, b, form=form), ref, 36, label=form)
    # the same events without the odd hit, in PAPER and CHAIN mode
    b = _block_tile_events(np.random.default_rng(42), 12, 3)
    for mode in (0, 1):
        ref = _oracle(oracle_mod, 3, mode, 0.25, 0.25, b)
        assert_same(gpu_select(_ctx(lib, 3, mode), b), ref, 36, label=f"mode={mode}")


def test_block_tile_station_block_finds_invalid_z(lib, oracle_mod):
    # z <= 0 in a non-trigger station of a block-tile event is found by that
    # station's own block: the whole run reports JPSI_EINVAL
    b = _block_tile_events(np.random.default_rng(43), 4, 3, odd_hit=(1.0, 1.0, -5.0))
    r = gpu_select(_ctx(lib, 3, 1), b)
    assert r["status"] == lib.JPSI_EINVAL


@pytest.mark.parametrize("mode", [0, 1])
def test_run_host_pinned_matches_oracle(lib, oracle_mod, synth_mod, mode):
    # pinned host buffers: PAPER mode reads the trigger station straight from
    # host memory over the link (no upload), CHAIN mode copies every station;
    # both equal the oracle, on log-normal events that reach every tile
    import torch
    n, S = 3000, 4
    b = synth_mod.generate("lognormal_timeslices", 0, n)
    assert np.diff(b["offsets"]).max() > 384  # some events run on the block tile
    ref = _oracle(oracle_mod, S, mode, 0.25, 0.25, b)
    pin = {k: torch.from_numpy(np.ascontiguousarray(b[k])).pin_memory() for k in ("x", "y", "z", "offsets")}
    acc = torch.zeros((n + 31) // 32, dtype=torch.int32).pin_memory()
    tc = torch.zeros(n, dtype=torch.int32).pin_memory()
    to = torch.zeros(n * S + 1, dtype=torch.int64).pin_memory()
    tr = torch.zeros((ref["trip_needed"] + 3, 3), dtype=torch.int32).pin_memory()
    o = lib.jpsi_outputs()
    o.accept_bits, o.track_counts, o.trip_off, o.triplets = acc.data_ptr(), tc.data_ptr(), to.data_ptr(), tr.data_ptr()
    o.trip_capacity = tr.shape[0]
    hb = lib.make_batch(pin["x"], pin["y"], pin["z"], pin["offsets"], n, b["n_hits"])
    ctx = _ctx(lib, S, mode)
    for _ in range(2):  # the second run reuses the context's buffers and graphs
        s = lib.jpsi_run_host(ctx.ctx, hb, o, 0)
        assert s == 0, lib.jpsi_strerror(s)
        host = {"status": 0, "trip_needed": o.trip_needed, "accept_bits": acc.numpy().view(np.uint32),
                "track_counts": tc.numpy(), "trip_off": to.numpy(), "triplets": tr.numpy()[: o.trip_needed]}
        assert_same(host, ref, n * S, label=f"mode={mode}")


def _z_table(w):
    """The workload's layer planes as a geometry table: station z + (l - 1) dz."""
    return np.array([np.float32(zs + (l - 1) * w.layer_dz) for zs in w.station_z for l in range(3)], np.float32)


def _check_planar(b, table, S):
    """Every hit of the generated batch lies on its layer's plane."""
    layer = np.repeat(np.tile(np.arange(3 * S), b["n_events"]), np.diff(b["offsets"]))
    assert np.array_equal(b["z"], table[layer])


@pytest.mark.parametrize("workload,n", [("poisson20_1k", 1000), ("lognormal_timeslices", 1500)])
def test_geometry_z_table_device(lib, synth_mod, workload, n):
    # z = NULL with a per-layer table: the library fills per-hit z on the
    # device and the results equal the run on the per-hit z array
    import torch
    w = synth_mod.WORKLOADS[workload]
    S = w.n_stations
    b = synth_mod.generate(w, 0, n)
    table = _z_table(w)
    _check_planar(b, table, S)
    ctx = _ctx(lib, S, 1)
    ref = gpu_select(ctx, b)
    d = {k: torch.from_numpy(b[k]).cuda() for k in ("x", "y", "offsets")}
    zt = torch.from_numpy(table).cuda()
    for form in ("plain", "batched"):
        r = ctx.select(d["x"], d["y"], None, d["offsets"], n, form=form, z_layer=zt)
        torch.cuda.synchronize()
        got = {"status": r["status"], "trip_needed": r["trip_needed"],
               "accept_bits": r["accept_bits"].cpu().numpy().view(np.uint32),
               "track_counts": r["track_counts"].cpu().numpy(), "trip_off": r["trip_off"].cpu().numpy(),
               "triplets": r["triplets"].cpu().numpy()}
        assert_same(got, ref, n * S, label=form)


@pytest.mark.parametrize("n", [2000, 140_000])
def test_geometry_z_table_host(lib, synth_mod, n):
    # jpsi_run_host with z = NULL: 8 bytes per hit uploaded and z filled on the
    # device (one piece, and per chunk on the pipelined path for >= 131072 events)
    w = synth_mod.WORKLOADS["poisson20_1k"]
    b = synth_mod.generate(w, 0, n)
    table = _z_table(w)
    _check_planar(b, table, 4)
    ctx = _ctx(lib)
    dev = gpu_select(ctx, b)
    acc = np.zeros((n + 31) // 32, np.uint32)
    tc = np.zeros(n, np.int32)
    to = np.zeros(n * 4 + 1, np.int64)
    tr = np.zeros((dev["trip_needed"] + 5, 3), np.int32)
    o = lib.jpsi_outputs()
    o.accept_bits, o.track_counts, o.trip_off, o.triplets = acc.ctypes.data, tc.ctypes.data, to.ctypes.data, tr.ctypes.data
    o.trip_capacity = len(tr)
    hb = lib.make_batch(b["x"], b["y"], None, b["offsets"], n, b["n_hits"], z_layer=table)
    for _ in range(2):
        s = lib.jpsi_run_host(ctx.ctx, hb, o, 0)
        assert s == 0, lib.jpsi_strerror(s)
        host = {"status": 0, "trip_needed": o.trip_needed, "accept_bits": acc, "track_counts": tc, "trip_off": to,
                "triplets": tr[: o.trip_needed]}
        assert_same(host, dev, n * 4)
    # no z and no table: refused
    hb = lib.make_batch(b["x"], b["y"], None, b["offsets"], n, b["n_hits"])
    assert lib.jpsi_run_host(ctx.ctx, hb, o, 0) == lib.JPSI_EINVAL


@pytest.mark.parametrize("ndf,minc,cuts", [(3, 2, (0.03, 0.025)), (3, 2, (0.25, 0.25)), (2, 1, (0.25, 0.25)),
                                           (2, 3, (0.25, 0.25)), (3, 0, (0.25, 0.25))])
def test_ndf_and_min_candidates(lib, oracle_mod, synth_mod, ndf, minc, cuts):
    # the degrees of freedom scale the cut (C = fl32(ndf * t)) and
    # min_candidates sets the accept threshold (Sec. 3.2 steps 2b and 3);
    # the paper's printed cuts are tried with ndf = 3 as well
    for wl, n in (("poisson20_1k", 1000), ("poisson100_1m", 3000)):
        b = synth_mod.generate(wl, 0, n)
        for mode in (0, 1):
            ref = oracle_mod.run(oracle_mod.params(4, mode, t_xz=cuts[0], t_yz=cuts[1], ndf=ndf, min_candidates=minc),
                                 b, n_threads=16)
            ctx = lib.Context(lib.params(4, mode, t_xz=cuts[0], t_yz=cuts[1], ndf=ndf, min_candidates=minc))
            for form in ("plain", "batched"):
                assert_same(gpu_select(ctx, b, form=form), ref, n * 4, label=f"{wl} mode={mode} {form}")
            ctx.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_distinct_hits(lib, oracle_mod, synth_mod, mode):
    # "at least two triplets" (Sec. 3.2 step 3) read as two candidates that
    # share no hit, on every path: small and medium tiles (Poisson(20),
    # log-normal), the block tile (dense trigger stations, split by station in
    # CHAIN mode), the unpruned kernel (a layer past the block tile) and hand
    # events whose candidates all share the middle-layer hit
    from helpers import shared_hit_event
    rng = np.random.default_rng(77)
    dense = []
    for _ in range(8):
        tx, ty = rng.uniform(-0.3, 0.3, 2)
        dense.append([[(tx * z + rng.normal(0, 0.05), ty * z + rng.normal(0, 0.05), z) for _ in range(9)]
                      for z in (120.0, 130.0, 140.0, 155.0, 165.0, 175.0)])
    huge = []
    for n in (2100, 2200):
        ev = []
        for li, z in enumerate((120.0, 130.0, 140.0, 155.0, 165.0, 175.0)):
            m = n if li == 4 else 30
            r = rng.uniform(15, 0.4 * z, m)
            ph = rng.uniform(0, 2 * np.pi, m)
            hits = [(float(a * np.cos(p)), float(a * np.sin(p)), z) for a, p in zip(r, ph)]
            hits += [(0.1 * z + 0.3 * q, -0.05 * z, z) for q in range(3)]
            ev.append(hits)
        huge.append(ev)
    shared = [shared_hit_event(2, False, dz=10.0, pitch=35.0) for _ in range(3)] + [shared_hit_event(2, True)]
    cases = [("poisson20_1k", synth_mod.generate("poisson20_1k", 0, 1000), 4, 0.25),
             ("lognormal", synth_mod.generate("lognormal_timeslices", 0, 2000), 4, 0.25),
             ("dense+huge+shared", make_batch(dense + huge + shared, 2), 2, 0.25)]
    for name, b, S, t in cases:
        ref = oracle_mod.run(oracle_mod.params(S, mode, t_xz=t, distinct_hits=1), b, n_threads=16)
        base = oracle_mod.run(oracle_mod.params(S, mode, t_xz=t), b, n_threads=16)
        assert ref["status"] == 0
        if name.startswith("dense"):  # the rule decides some events here
            assert not np.array_equal(ref["accept_bits"], base["accept_bits"])
        ctx = lib.Context(lib.params(S, mode, t_xz=t, distinct_hits=1))
        for form in ("plain", "batched"):
            assert_same(gpu_select(ctx, b, form=form), ref, b["n_events"] * S, label=f"{name} mode={mode} {form}")
        ctx.close()


def test_distinct_hits_parameters(lib):
    import ctypes
    for minc, ok in ((0, True), (1, True), (2, True), (3, False)):
        p = lib.params(4, 1, min_candidates=minc, distinct_hits=1)
        if ok:
            lib.Context(p).close()
        else:
            with pytest.raises(lib.JpsiError):
                lib.Context(p)
    with pytest.raises(lib.JpsiError):
        lib.Context(lib.params(4, 1, distinct_hits=2))
