"""Error paths under host-side fault injection (jpsi_inject_fault): a failed
device allocation returns JPSI_ENOMEM and leaves the context usable, and a
serving slot repeats a failed run once.  Nothing is injected on the GPU."""
import numpy as np
import pytest

from gpu_helpers import assert_same, gpu_select, to_device
from helpers import sorted_triplets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1810_11966_gb300 as jp
    jp.load(build_if_missing=True)
    return jp


def test_inject_fault_arguments(lib):
    ctx = lib.Context(lib.params(4, 1))
    assert lib.jpsi_inject_fault(ctx.ctx, lib.FAULT_ALLOC, -1) == lib.JPSI_EINVAL
    assert lib.jpsi_inject_fault(ctx.ctx, 7, 1) == lib.JPSI_EINVAL
    assert lib.jpsi_inject_fault(None, lib.FAULT_RUN, 1) == lib.JPSI_EINVAL
    assert lib.jpsi_inject_fault(ctx.ctx, lib.FAULT_RUN, 0) == lib.JPSI_OK


def test_failed_allocation_then_recovery(lib, synth_mod, oracle_mod):
    b = synth_mod.generate("lognormal_timeslices", 0, 3000)
    ref = oracle_mod.run(oracle_mod.params(4, 1, t_xz=0.25), b, n_threads=8)
    ctx = lib.Context(lib.params(4, 1, t_xz=0.25))
    # a fresh context grows its scratch on the first run: that allocation fails
    assert lib.jpsi_inject_fault(ctx.ctx, lib.FAULT_ALLOC, 1) == 0
    d = to_device(b)
    r = ctx.select(d["x"], d["y"], d["z"], d["offsets"], d["n_events"], capacity=0)
    assert r["status"] == lib.JPSI_ENOMEM and "injected" in r["error"]
    # the fault is spent: the same context now runs, with exact results
    for form in ("batched", "plain"):
        assert_same(gpu_select(ctx, b, form=form), ref, b["n_events"] * 4, label=form)


def _host_out(lib, n, S, cap):
    out = {"acc": np.zeros((n + 31) // 32, np.uint32), "tc": np.zeros(n, np.int32),
           "toff": np.zeros(n * S + 1, np.int64), "trip": np.zeros((max(cap, 1), 3), np.int32)}
    o = lib.jpsi_outputs()
    o.accept_bits, o.track_counts = out["acc"].ctypes.data, out["tc"].ctypes.data
    o.trip_off, o.triplets, o.trip_capacity = out["toff"].ctypes.data, out["trip"].ctypes.data, max(cap, 1)
    return o, out


def test_serving_repeats_a_failed_run_once(lib, synth_mod, oracle_mod):
    S = 4
    b = synth_mod.generate("lognormal_timeslices", 0, 1500)
    ref = oracle_mod.run(oracle_mod.params(S, 1, t_xz=0.25), b, n_threads=8)
    cap = int(ref["trip_needed"])
    ctx = lib.Context(lib.params(S, 1, t_xz=0.25))
    assert lib.jpsi_serve_start(ctx.ctx, 2, b["n_events"], b["n_hits"], cap) == 0
    hb = lib.make_batch(b["x"], b["y"], b["z"], b["offsets"], b["n_events"], b["n_hits"])
    n_units = b["n_events"] * S
    ref_rows = sorted_triplets(ref["trip_off"], ref["triplets"], n_units)

    def serve(n_faults):
        assert lib.jpsi_inject_fault(ctx.ctx, lib.FAULT_RUN, n_faults) == 0
        o, out = _host_out(lib, b["n_events"], S, cap)
        s, t = lib.jpsi_serve_submit(ctx.ctx, hb, o)
        assert s == 0
        ws, rs, _ = lib.jpsi_serve_wait(ctx.ctx, t, 60000)
        assert ws == 0
        return rs, o, out

    # one failure: the slot's second attempt runs, and its result is exact
    rs, o, out = serve(1)
    assert rs == lib.JPSI_OK and o.trip_needed == ref["trip_needed"]
    assert np.array_equal(out["acc"], ref["accept_bits"]) and np.array_equal(out["tc"], ref["track_counts"])
    assert np.array_equal(sorted_triplets(out["toff"], out["trip"][:cap], n_units), ref_rows)
    # two failures: the second attempt fails too, and that is reported
    rs, _, _ = serve(2)
    assert rs == lib.JPSI_ECUDA
    # nothing is left over: the next request is served normally
    rs, o, out = serve(0)
    assert rs == lib.JPSI_OK and np.array_equal(out["tc"], ref["track_counts"])
    assert lib.jpsi_serve_stop(ctx.ctx) == 0
