"""Free-streaming selection on the GPU (jpsi_run_stream, jpsi_run_stream_plain)
against the oracle's free-streaming selection, bit-exact.

The rule (include/jpsi.h): a triplet counts only when its hits are
coincident, max t <= fl32(min t + dt), and it belongs to the window holding
its earliest time; CHAIN partners are coincident passing triplets anywhere in
the timeslice whose six hits with the trigger triplet are coincident.  The
library builds one event per window on the device and runs the selection
kernels with the time tests compiled in; these tests cover every tile (by
the tuning cutoffs), both forms, the emit fallback, the edge cases and the
refusals, and the full-size timeslice on sampled windows.
"""
import numpy as np
import pytest

from gpu_helpers import assert_same, gpu_select_stream
from helpers import accept_list, sorted_triplets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1810_11966_gb300 as jp
    jp.load(build_if_missing=True)
    return jp


def _ctx(lib, S, mode, t=0.25, **knobs):
    ctx = lib.Context(lib.params(S, mode, t_xz=t))
    if knobs:
        tu = lib.jpsi_get_tuning(ctx.ctx)
        for k, v in knobs.items():
            setattr(tu, k, v)
        assert lib.jpsi_set_tuning(ctx.ctx, tu) == lib.JPSI_OK, ctx.last_error()
    return ctx


def _ref(oracle_mod, S, mode, ts, bounds=None, dt=None, t=0.25):
    p = oracle_mod.params(S, mode, t_xz=t, t_yz=t)
    return oracle_mod.stream(p, ts, ts["bounds"] if bounds is None else bounds, ts["dt"] if dt is None else dt)


@pytest.fixture(scope="module")
def small_ts(synth_mod):
    # 400 collisions of the 20-hits-per-layer recipe at 1e7/s, 100 ns windows
    return synth_mod.timeslice("poisson20_1k", 0, 400, window_ns=100.0, dt_ns=15.0)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("form", ["batched", "plain"])
def test_stream_matches_oracle(lib, oracle_mod, small_ts, mode, form):
    ref = _ref(oracle_mod, 4, mode, small_ts)
    K = len(small_ts["bounds"]) - 1
    assert ref["status"] == 0 and ref["trip_needed"] > 0 and accept_list(ref["accept_bits"], K).any()
    ctx = _ctx(lib, 4, mode)
    g = gpu_select_stream(ctx, small_ts, form=form)
    assert_same(g, ref, K * 4, label=f"{form} mode {mode}")
    ctx.close()


@pytest.mark.parametrize("window_ns,dt_ns", [(50.0, 40.0), (300.0, 5.0), (100.0, 0.0)])
def test_stream_windows_and_widths(lib, oracle_mod, synth_mod, window_ns, dt_ns):
    # short windows with a wide coincidence (many triplets across
    # boundaries), long windows with a narrow one, and dt = 0
    ts = synth_mod.timeslice("poisson20_1k", 1000, 250, window_ns=window_ns, dt_ns=dt_ns)
    K = len(ts["bounds"]) - 1
    for mode in (0, 1):
        ref = _ref(oracle_mod, 4, mode, ts)
        ctx = _ctx(lib, 4, mode)
        for form in ("batched", "plain"):
            assert_same(gpu_select_stream(ctx, ts, form=form), ref, K * 4, label=f"{window_ns} {dt_ns} {form}")
        ctx.close()


@pytest.mark.parametrize("caps", [(16, 40), (32, 384), (1, 1)])
def test_stream_every_tile(lib, oracle_mod, synth_mod, caps):
    # lower layer cutoffs send windows to the medium warp tile and the block
    # tile; 300 ns windows hold ~3 collisions (~60 hits a layer)
    ts = synth_mod.timeslice("poisson20_1k", 2000, 300, window_ns=300.0, dt_ns=15.0)
    K = len(ts["bounds"]) - 1
    ref = _ref(oracle_mod, 4, 1, ts)
    ctx = _ctx(lib, 4, 1, small_layer_cap=caps[0], medium_layer_cap=caps[1])
    for form in ("batched", "plain"):
        assert_same(gpu_select_stream(ctx, ts, form=form), ref, K * 4, label=f"{caps} {form}")
    ctx.close()


def test_stream_emit_fallback(lib, oracle_mod, synth_mod):
    # record_cap = 0: triplet rows by the re-enumeration kernels
    ts = synth_mod.timeslice("poisson20_1k", 3000, 300, window_ns=200.0, dt_ns=15.0)
    K = len(ts["bounds"]) - 1
    ref = _ref(oracle_mod, 4, 1, ts)
    for caps in ((192, 384), (16, 40), (1, 1)):
        ctx = _ctx(lib, 4, 1, record_cap=0, small_layer_cap=caps[0], medium_layer_cap=caps[1])
        for form in ("batched", "plain"):
            assert_same(gpu_select_stream(ctx, ts, form=form), ref, K * 4, label=f"emit {caps} {form}")
        ctx.close()


def _huge_layer_timeslice(rng):
    """Two stations; window 1 has a layer of 2300 hits (past the block tile:
    the unpruned kernel) around a straight track; times within a few ns."""
    zl = [120.0, 130.0, 140.0, 155.0, 165.0, 175.0]
    groups = [[] for _ in range(6)]
    for c, (t0, big) in enumerate(((100.0, 0), (1100.0, 2300), (2100.0, 0))):
        tx, ty = rng.uniform(-0.2, 0.2, 2)
        for g, z in enumerate(zl):
            m = big if (g == 1 and big) else 25
            r = rng.uniform(15, 0.4 * z, m)
            ph = rng.uniform(0, 2 * np.pi, m)
            pts = [(float(a * np.cos(p)), float(a * np.sin(p))) for a, p in zip(r, ph)]
            pts += [(tx * z + rng.normal(0, 0.03), ty * z + rng.normal(0, 0.03)) for _ in range(2)]
            for x, y in pts:
                groups[g].append((np.float32(t0 + rng.uniform(0, 6)), x, y, z))
    xs, ys, zs, ts, off = [], [], [], [], [0]
    for g in range(6):
        for t, x, y, z in sorted(groups[g], key=lambda r: r[0]):
            ts.append(t), xs.append(x), ys.append(y), zs.append(z)
        off.append(len(xs))
    return {"x": np.array(xs, np.float32), "y": np.array(ys, np.float32), "z": np.array(zs, np.float32),
            "t": np.array(ts, np.float32), "offsets": np.array(off, np.int32),
            "bounds": np.array([0.0, 1000.0, 2000.0, 3000.0], np.float32), "dt": 10.0}


@pytest.mark.parametrize("mode", [0, 1])
def test_stream_unpruned_window(lib, oracle_mod, mode):
    ts = _huge_layer_timeslice(np.random.default_rng(11))
    ref = _ref(oracle_mod, 2, mode, ts)
    assert ref["trip_needed"] > 0
    for rc in (-1, 0):
        ctx = _ctx(lib, 2, mode, record_cap=rc)
        for form in ("batched", "plain"):
            assert_same(gpu_select_stream(ctx, ts, form=form), ref, 3 * 2, label=f"{form} {rc}")
        ctx.close()


def test_stream_edge_cases(lib, oracle_mod, small_ts):
    ctx = _ctx(lib, 4, 1)
    S = 4
    # no windows
    g = gpu_select_stream(ctx, small_ts, bounds=small_ts["bounds"][:1])
    assert g["status"] == 0 and g["trip_needed"] == 0 and list(g["trip_off"]) == [0]
    # windows before and after every hit, and an empty timeslice
    far = np.array([-5000.0, -4000.0, -3000.0], np.float32)
    g = gpu_select_stream(ctx, small_ts, bounds=far)
    assert g["status"] == 0 and g["trip_needed"] == 0 and not g["track_counts"].any()
    empty = {"x": np.zeros(0, np.float32), "y": np.zeros(0, np.float32), "z": np.zeros(0, np.float32),
             "t": np.zeros(0, np.float32), "offsets": np.zeros(3 * S + 1, np.int32),
             "bounds": np.array([0.0, 10.0, 20.0], np.float32), "dt": 5.0}
    g = gpu_select_stream(ctx, empty)
    assert g["status"] == 0 and g["trip_needed"] == 0 and list(g["trip_off"]) == [0] * 9
    # a per-layer z table gives the same results as per-hit z
    table = np.unique(small_ts["z"])
    assert len(table) == 3 * S
    a = gpu_select_stream(ctx, small_ts)
    b = gpu_select_stream(ctx, small_ts, z_layer=np.sort(table))
    ref = _ref(oracle_mod, 4, 1, small_ts)
    K = len(small_ts["bounds"]) - 1
    assert_same(a, ref, K * S)
    assert_same(b, ref, K * S, label="z table")
    # event runs and stream runs alternate on one context (graphs re-captured)
    import paper_1810_11966_gb300 as jp  # noqa: F401
    from gpu_helpers import gpu_select
    import synth
    ev = synth.generate("poisson20_1k", 0, 300)
    er = oracle_mod.run(oracle_mod.params(4, 1, t_xz=0.25, t_yz=0.25), ev)
    assert_same(gpu_select(ctx, ev), er, 300 * S, label="event run after stream")
    assert_same(gpu_select_stream(ctx, small_ts), ref, K * S, label="stream after event run")
    ctx.close()


def test_stream_refusals(lib, small_ts):
    ctx = _ctx(lib, 4, 1)
    E = lib.JPSI_EINVAL

    def run(mod=None, bounds=None, dt=None):
        ts = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in small_ts.items()}
        if mod:
            mod(ts)
        return gpu_select_stream(ctx, ts, bounds=bounds, dt=dt)["status"]

    off = small_ts["offsets"]

    def unsort(ts):
        a = off[5] + 3
        ts["t"][a], ts["t"][a + 1] = ts["t"][a + 1] + 1.0, ts["t"][a]

    def nan_t(ts):
        ts["t"][off[7] + 2] = np.nan

    def z_zero(ts):
        ts["z"][off[1] + 4] = 0.0

    def bad_off(ts):
        ts["offsets"][3], ts["offsets"][4] = ts["offsets"][4], ts["offsets"][3]

    for m in (unsort, nan_t, z_zero, bad_off):
        assert run(m) == E, m.__name__
    b = small_ts["bounds"].copy()
    b[5] = b[4]
    assert run(bounds=b) == E
    b = small_ts["bounds"].copy()
    b[7] = np.nan
    assert run(bounds=b) == E
    assert run(dt=-1.0) == E
    assert run(dt=float("inf")) == E
    # the context still works afterwards
    assert run() == 0
    ctx.close()
    # PAPER mode reads only the trigger station: z <= 0 elsewhere is legal
    pap = _ctx(lib, 4, 0)
    ts = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in small_ts.items()}
    ts["z"][off[1] + 4] = 0.0
    assert gpu_select_stream(pap, ts)["status"] == 0
    pap.close()
    # distinct_hits has no free-streaming definition
    d = lib.Context(lib.params(4, 1, t_xz=0.25, distinct_hits=1))
    assert gpu_select_stream(d, small_ts)["status"] == E
    d.close()


def test_stream_full_size_sampled(lib, oracle_mod, synth_mod):
    # the 100 000-collision timeslice (10 ms at 1e7 collisions/s) in the
    # batched form with the autotuned shape; the oracle computes sampled
    # windows (each through the whole timeslice, so partners may lie in
    # neighbouring windows) and every window is checked for consistency
    ts = synth_mod.timeslice("poisson100_stream")
    S, K = 4, len(ts["bounds"]) - 1
    ctx = _ctx(lib, S, 1)
    g = gpu_select_stream(ctx, ts)
    assert g["status"] == 0, g["error"]
    to, tc = g["trip_off"], g["track_counts"]
    uc = np.diff(to).reshape(K, S)
    assert (uc >= 0).all() and to[0] == 0 and to[-1] == g["trip_needed"]
    assert (tc <= uc[:, S - 1]).all()
    assert np.array_equal(accept_list(g["accept_bits"], K), tc >= 2)
    assert accept_list(g["accept_bits"], K).sum() > 0
    rows = g["triplets"]
    gs = np.diff(ts["offsets"])
    unit = np.repeat(np.arange(K * S), np.diff(to))
    st = unit % S
    for l in range(3):
        assert (rows[:, l] >= 0).all() and (rows[:, l] < gs[3 * st + l]).all()
    rng = np.random.default_rng(8)
    dense = int(np.argmax(uc.sum(axis=1)))
    picks = sorted(set([0, K - 1, dense] + [int(v) for v in rng.integers(0, K, 5)] +
                       [int(np.nonzero(tc >= 2)[0][0])]))
    p = oracle_mod.params(S, 1, t_xz=0.25, t_yz=0.25)
    for k in picks:
        r = oracle_mod.stream(p, ts, ts["bounds"][k:k + 2], ts["dt"])
        assert r["status"] == 0
        assert r["track_counts"][0] == tc[k], k
        assert accept_list(r["accept_bits"], 1)[0] == accept_list(g["accept_bits"], K)[k], k
        assert np.array_equal(np.diff(r["trip_off"]), uc[k]), k
        mine = rows[to[k * S]:to[(k + 1) * S]]
        got = sorted_triplets(to[k * S:(k + 1) * S + 1] - to[k * S], mine, S)
        assert np.array_equal(got, sorted_triplets(r["trip_off"], r["triplets"], S)), k
    ctx.close()
