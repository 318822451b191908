"""Full-size parity: the 10^6-event Poisson(100) workload through jpsi_run in
the launch configuration bench.py times, checked on sampled event ranges that
the oracle computes on their own (the generator reproduces any event range
exactly), and the 2 000-event subset of the 6-station stress workload."""
import numpy as np
import pytest

from helpers import accept_list, sorted_triplets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1810_11966_gb300 as jp
    jp.load(build_if_missing=True)
    return jp


def test_million_events_sampled(lib, oracle_mod, synth_mod):
    import torch
    w = synth_mod.WORKLOADS["poisson100_1m"]
    n, S = w.n_events, w.n_stations
    b = synth_mod.generate(w)
    d = {k: torch.from_numpy(b[k]).cuda() for k in ("x", "y", "z", "offsets")}
    ctx = lib.Context(lib.params(S, 1, t_xz=0.25), hbm_budget=64 << 30)
    r = ctx.select(d["x"], d["y"], d["z"], d["offsets"], n)
    assert r["status"] == 0
    tc = r["track_counts"].cpu().numpy()
    acc = accept_list(r["accept_bits"].cpu().numpy().view(np.uint32), n)
    toff = r["trip_off"].cpu().numpy()
    trip = r["triplets"].cpu().numpy()
    del d, b
    # events near the start, the middle, the end, and a ragged tail
    for e0, m in ((0, 600), (371_113, 700), (999_000, 1000), (640_001, 333)):
        sub = synth_mod.generate(w, e0, m)
        ref = oracle_mod.run(oracle_mod.params(S, 1, t_xz=0.25), sub, n_threads=16)
        assert np.array_equal(tc[e0:e0 + m], ref["track_counts"])
        assert np.array_equal(acc[e0:e0 + m], accept_list(ref["accept_bits"], m))
        u0, u1 = e0 * S, (e0 + m) * S
        got_off = toff[u0:u1 + 1] - toff[u0]
        assert np.array_equal(got_off, ref["trip_off"])
        got = trip[toff[u0]:toff[u1]]
        assert np.array_equal(sorted_triplets(got_off, got, m * S),
                              sorted_triplets(ref["trip_off"], ref["triplets"], m * S))
    # totals that hold at any size
    assert toff[-1] == r["trip_needed"] == len(trip)
    assert np.all(np.diff(toff) >= 0)
    assert np.all((acc == (tc >= 2)))


@pytest.mark.slow
def test_stress_2000_events(lib, oracle_mod, synth_mod):
    w = synth_mod.WORKLOADS["poisson1500_6st"]
    b = synth_mod.generate(w, 0, 2000)
    ref = oracle_mod.run(oracle_mod.params(6, 1, t_xz=1.0), b, n_threads=16)
    from gpu_helpers import assert_same, gpu_select
    ctx = lib.Context(lib.params(6, 1, t_xz=1.0), hbm_budget=32 << 30)
    g = gpu_select(ctx, b)
    assert_same(g, ref, 2000 * 6)
    assert ref["trip_needed"] > 2000 * 6 * 1000
