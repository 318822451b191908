"""Every execution path of the library against the oracle, bit-exact.

The tuning knobs (include/jpsi.h, jpsi_set_tuning) move events between the
warp tiles, the block tile and the unpruned kernel, and switch the triplet
rows from the scatter of recorded entries to the re-enumeration (emit)
kernels.  None of them may change a result; these tests force each path.
"""
import numpy as np
import pytest

from gpu_helpers import assert_same, gpu_select
from helpers import make_batch

pytestmark = pytest.mark.gpu

# kernel launches of one run with triplet rows.  Batched: counting (1 + 10),
# then the scatter (1) or the emit fallback (4).  One-launch form: the warp
# grid, the block grid and the tail (1 + 1 + 4), then the scatter (1) or the
# two grids again (2).
LAUNCHES = {("batched", "scatter"): 12, ("batched", "emit"): 15, ("plain", "scatter"): 7, ("plain", "emit"): 8}


@pytest.fixture(scope="module")
def lib():
    import paper_1810_11966_gb300 as jp
    jp.load(build_if_missing=True)
    return jp


def _oracle(oracle_mod, S, mode, t, batch, threads=16):
    return oracle_mod.run(oracle_mod.params(S, mode, t_xz=t, t_yz=t), batch, n_threads=threads)


def _tuned(lib, S, mode, t=0.25, **knobs):
    ctx = lib.Context(lib.params(S, mode, t_xz=t))
    tu = lib.jpsi_get_tuning(ctx.ctx)
    for k, v in knobs.items():
        setattr(tu, k, v)
    assert lib.jpsi_set_tuning(ctx.ctx, tu) == lib.JPSI_OK, ctx.last_error()
    return ctx


def _launches(lib, ctx, batch, form, capacity):
    """Kernel launches of one timed run with triplet rows (capacity known)."""
    lib.jpsi_timing_enable(ctx.ctx, True)
    g = gpu_select(ctx, batch, form=form, capacity=capacity)
    t = lib.jpsi_timing_get(ctx.ctx)
    lib.jpsi_timing_enable(ctx.ctx, False)
    assert t.runs == 1
    return g, t.kernel_launches


def _dense_and_huge_events(rng):
    """Two stations: events whose trigger station holds more passing
    triplets than a warp keeps (block tile), and events with a layer past the
    block tile (unpruned kernel)."""
    zl = [120.0, 130.0, 140.0, 155.0, 165.0, 175.0]
    events = []
    for _ in range(6):
        tx, ty = rng.uniform(-0.3, 0.3, 2)
        events.append([[(tx * z + rng.normal(0, 0.05), ty * z + rng.normal(0, 0.05), z) for _ in range(9)]
                       for z in zl])
    for n in (2100, 2300):
        ev = []
        for li, z in enumerate(zl):
            m = n if li == 1 else 30
            r = rng.uniform(15, 0.4 * z, m)
            ph = rng.uniform(0, 2 * np.pi, m)
            hits = [(float(a * np.cos(p)), float(a * np.sin(p)), z) for a, p in zip(r, ph)]
            hits.append((0.1 * z, -0.05 * z, z))
            ev.append(hits)
        events.append(ev)
    return make_batch(events, 2)


@pytest.mark.parametrize("mode", [0, 1])
def test_emit_fallback_on_every_path(lib, oracle_mod, synth_mod, mode):
    # record_cap = 0: the counting pass records nothing, so the rows of every
    # path (small and medium warp tiles, block tile, unpruned kernel) come
    # from the emit kernels; the launch count shows which phase ran
    cases = [("poisson100_1m", synth_mod.generate("poisson100_1m", 0, 2000), 4),
             ("lognormal_timeslices", synth_mod.generate("lognormal_timeslices", 0, 2500), 4),
             ("dense+huge", _dense_and_huge_events(np.random.default_rng(5)), 2)]
    for name, b, S in cases:
        ref = _oracle(oracle_mod, S, mode, 0.25, b)
        assert ref["trip_needed"] > 0
        for form in ("plain", "batched"):
            emit = _tuned(lib, S, mode, record_cap=0)
            g, n = _launches(lib, emit, b, form, ref["trip_needed"])
            assert_same(g, ref, b["n_events"] * S, label=f"{name} {form} emit")
            assert n == LAUNCHES[form, "emit"], (name, form, n)
            emit.close()
            scat = _tuned(lib, S, mode)
            gpu_select(scat, b, form=form, capacity=ref["trip_needed"])  # sizes the record
            g, n = _launches(lib, scat, b, form, ref["trip_needed"])
            assert_same(g, ref, b["n_events"] * S, label=f"{name} {form} scatter")
            assert n == LAUNCHES[form, "scatter"], (name, form, n)
            scat.close()


def test_record_overflow_falls_back(lib, oracle_mod, synth_mod):
    # a record smaller than the run's triplets overflows: rows by the emit
    # kernels, same result
    b = synth_mod.generate("lognormal_timeslices", 0, 1500)
    ref = _oracle(oracle_mod, 4, 1, 0.25, b)
    ctx = _tuned(lib, 4, 1, record_cap=max(ref["trip_needed"] // 3, 1))
    for _ in range(2):
        g, n = _launches(lib, ctx, b, "batched", ref["trip_needed"])
        assert_same(g, ref, 6000)
        assert n == LAUNCHES["batched", "emit"]


@pytest.mark.parametrize("caps", [(32, 384), (192, 200), (16, 40), (192, 384)])
def test_layer_cutoffs_move_events_not_results(lib, oracle_mod, synth_mod, caps):
    # lowering the warp tiles' layer cutoffs sends events to the medium warp
    # tile and the block tile; results stay the oracle's
    b = synth_mod.generate("poisson100_1m", 100, 1500)
    ref = _oracle(oracle_mod, 4, 1, 0.25, b)
    ctx = _tuned(lib, 4, 1, small_layer_cap=caps[0], medium_layer_cap=caps[1])
    for form in ("plain", "batched"):
        assert_same(gpu_select(ctx, b, form=form), ref, 6000, label=f"{caps} {form}")


def test_tuning_rejects_bad_values(lib):
    ctx = lib.Context(lib.params(4, 1))
    good = lib.jpsi_get_tuning(ctx.ctx)
    assert good.as_dict() == {"light_wpb": 4, "light_grab": 2, "small_layer_cap": 192, "medium_layer_cap": 384,
                              "heavy_ctas_per_sm": 0, "record_cap": -1}
    for field, bad in [("light_wpb", 3), ("light_grab", 0), ("light_grab", 65), ("small_layer_cap", 193),
                       ("medium_layer_cap", 0), ("heavy_ctas_per_sm", -1), ("heavy_ctas_per_sm", 99),
                       ("record_cap", -2), ("reserved", 1)]:
        t = lib.jpsi_get_tuning(ctx.ctx)
        setattr(t, field, bad)
        assert lib.jpsi_set_tuning(ctx.ctx, t) == lib.JPSI_EINVAL, field
        assert lib.jpsi_get_tuning(ctx.ctx).as_dict() == good.as_dict()


def test_autotune_reports_its_choice(lib, synth_mod):
    import torch
    b = synth_mod.generate("lognormal_timeslices", 0, 3000)
    ctx = lib.Context(lib.params(4, 1))
    ref = gpu_select(ctx, b)
    d = {k: torch.from_numpy(b[k]).cuda() for k in ("x", "y", "z", "offsets")}
    assert lib.jpsi_autotune(ctx.ctx, lib.make_batch(d["x"], d["y"], d["z"], d["offsets"], 3000)) == 0
    t = lib.jpsi_get_tuning(ctx.ctx)
    assert t.light_wpb in (2, 4, 8) and t.small_layer_cap in (96, 128, 160, 192)
    assert t.medium_layer_cap in (256, 320, 384) and t.record_cap == -1
    tm = lib.jpsi_timing_get(ctx.ctx)
    assert (tm.light_wpb, tm.light_grab) == (t.light_wpb, t.light_grab)
    assert_same(gpu_select(ctx, b), ref, 12000)


@pytest.mark.parametrize("record_cap", [-1, 0])
def test_run_host_pipelined_lognormal(lib, oracle_mod, synth_mod, record_cap):
    # >= 131072 CHAIN events: jpsi_run_host counts them chunk by chunk while
    # the next chunk uploads.  Log-normal events reach the medium and block
    # tiles in every chunk; with record_cap = 0 the rows come from the emit
    # kernels over the whole batch, which must see every chunk's events.
    n, S = 140_000, 4
    b = synth_mod.generate("lognormal_timeslices", 0, n)
    per_layer = np.diff(b["offsets"]).reshape(n, 3 * S).max(axis=1)
    first = per_layer[: n // 4]
    assert (first > 384).sum() > 50 and ((first > 192) & (first <= 384)).sum() > 500
    ref = _oracle(oracle_mod, S, 1, 0.25, b)
    ctx = _tuned(lib, S, 1, record_cap=record_cap)
    acc = np.zeros((n + 31) // 32, np.uint32)
    tc = np.zeros(n, np.int32)
    to = np.zeros(n * S + 1, np.int64)
    tr = np.zeros((ref["trip_needed"] + 1, 3), np.int32)
    o = lib.jpsi_outputs()
    o.accept_bits, o.track_counts, o.trip_off, o.triplets = acc.ctypes.data, tc.ctypes.data, to.ctypes.data, tr.ctypes.data
    o.trip_capacity = len(tr)
    hb = lib.make_batch(b["x"], b["y"], b["z"], b["offsets"], n)
    for _ in range(2):
        tr[:] = -1
        s = lib.jpsi_run_host(ctx.ctx, hb, o, 0)
        assert s == 0, ctx.last_error()
        host = {"status": 0, "trip_needed": o.trip_needed, "accept_bits": acc, "track_counts": tc, "trip_off": to,
                "triplets": tr[: o.trip_needed]}
        assert_same(host, ref, n * S, label=f"record_cap={record_cap}")
