"""Serving (continuous batching through jpsi_serve_*): every result is the
same as the same batch run alone, requests beyond the slot count wait for a
free slot, and waits are bounded."""
import threading

import numpy as np
import pytest

from helpers import sorted_triplets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1810_11966_gb300 as jp
    jp.load(build_if_missing=True)
    return jp


def _host_out(lib, n, S, cap):
    out = {"acc": np.zeros((n + 31) // 32, np.uint32), "tc": np.zeros(n, np.int32),
           "toff": np.zeros(n * S + 1, np.int64), "trip": np.zeros((max(cap, 1), 3), np.int32)}
    o = lib.jpsi_outputs()
    o.accept_bits, o.track_counts = out["acc"].ctypes.data, out["tc"].ctypes.data
    o.trip_off, o.triplets, o.trip_capacity = out["toff"].ctypes.data, out["trip"].ctypes.data, max(cap, 1)
    return o, out


def test_served_results_equal_solo(lib, synth_mod, oracle_mod):
    S = 4
    batches = [synth_mod.generate("lognormal_timeslices", e0, n) for e0, n in
               ((0, 700), (700, 1500), (2200, 300), (2500, 2000), (4500, 900), (5400, 1200), (6600, 50))]
    ctx = lib.Context(lib.params(S, 1, t_xz=0.25))
    solo = []
    for b in batches:
        o, out = _host_out(lib, b["n_events"], S, 200000)
        hb = lib.make_batch(b["x"], b["y"], b["z"], b["offsets"], b["n_events"], b["n_hits"])
        assert lib.jpsi_run_host(ctx.ctx, hb, o, 0) == 0
        out["n"] = o.trip_needed
        solo.append(out)
        # and the oracle agrees with the solo run
        ref = oracle_mod.run(oracle_mod.params(S, 1, t_xz=0.25), b, n_threads=8)
        assert np.array_equal(ref["track_counts"], out["tc"]) and ref["trip_needed"] == o.trip_needed
    max_ev = max(b["n_events"] for b in batches)
    max_hits = max(b["n_hits"] for b in batches)
    max_trip = max(s["n"] for s in solo)
    assert lib.jpsi_serve_start(ctx.ctx, 3, max_ev, max_hits, max_trip) == 0
    served = [None] * len(batches)
    keep = []
    tickets = [None] * len(batches)

    def submit_all():
        for i, b in enumerate(batches):  # 7 requests, 3 slots: submit blocks until one frees up
            o, out = _host_out(lib, b["n_events"], S, max_trip)
            hb = lib.make_batch(b["x"], b["y"], b["z"], b["offsets"], b["n_events"], b["n_hits"])
            keep.append((o, hb))
            s, t = lib.jpsi_serve_submit(ctx.ctx, hb, o)
            assert s == 0
            served[i] = (out, o)
            tickets[i] = t

    th = threading.Thread(target=submit_all)
    th.start()
    for i in range(len(batches)):
        while tickets[i] is None:
            th.join(0.001)
        ws, rs, lat = lib.jpsi_serve_wait(ctx.ctx, tickets[i], 60000)
        assert ws == 0 and rs == 0 and lat > 0
    th.join()
    for i, b in enumerate(batches):
        out, o = served[i]
        ref = solo[i]
        n_units = b["n_events"] * S
        assert o.trip_needed == ref["n"]
        assert np.array_equal(out["acc"], ref["acc"]) and np.array_equal(out["tc"], ref["tc"])
        assert np.array_equal(out["toff"], ref["toff"])
        assert np.array_equal(sorted_triplets(out["toff"], out["trip"][: ref["n"]], n_units),
                              sorted_triplets(ref["toff"], ref["trip"][: ref["n"]], n_units))
    # a ticket that never completes: the wait is bounded
    ws, _, _ = lib.jpsi_serve_wait(ctx.ctx, 10 ** 9, 50)
    assert ws == lib.JPSI_ETIMEOUT
    assert lib.jpsi_serve_stop(ctx.ctx) == 0
    s, _ = lib.jpsi_serve_submit(ctx.ctx, keep[0][1], keep[0][0])
    assert s == lib.JPSI_EINVAL


def test_serving_rejects_oversized_request(lib, synth_mod):
    b = synth_mod.generate("poisson20_1k", 0, 100)
    ctx = lib.Context(lib.params(4, 1))
    assert lib.jpsi_serve_start(ctx.ctx, 2, 50, 100000, 1000) == 0
    o, _ = _host_out(lib, 100, 4, 1000)
    hb = lib.make_batch(b["x"], b["y"], b["z"], b["offsets"], 100, b["n_hits"])
    s, _ = lib.jpsi_serve_submit(ctx.ctx, hb, o)
    assert s == lib.JPSI_EINVAL
    assert lib.jpsi_serve_stop(ctx.ctx) == 0


@pytest.mark.parametrize("batch_on,out_on", [("cuda", "cuda"), ("cuda", "cpu"), ("cpu", "cuda")])
def test_serving_device_batch_and_outputs(lib, synth_mod, oracle_mod, batch_on, out_on):
    # a batch and outputs in device memory of the context's device are used
    # in place; with either of them in host memory the slot copies; every
    # result equals the oracle's
    import torch
    S = 4
    b = synth_mod.generate("lognormal_timeslices", 0, 1200)
    ref = oracle_mod.run(oracle_mod.params(S, 1, t_xz=0.25), b, n_threads=8)
    cap = int(ref["trip_needed"])
    n, nu = b["n_events"], b["n_events"] * S
    ctx = lib.Context(lib.params(S, 1, t_xz=0.25))
    assert lib.jpsi_serve_start(ctx.ctx, 2, n, b["n_hits"], cap) == 0
    pin = out_on == "cpu"

    def put(a):
        return a.cuda() if batch_on == "cuda" else a.pin_memory()

    d = {k: put(torch.from_numpy(b[k])) for k in ("x", "y", "z", "offsets")}
    hb = lib.make_batch(d["x"], d["y"], d["z"], d["offsets"], n, b["n_hits"])
    acc = torch.zeros((n + 31) // 32, dtype=torch.int32, device=out_on, pin_memory=pin)
    tc = torch.zeros(n, dtype=torch.int32, device=out_on, pin_memory=pin)
    toff = torch.zeros(nu + 1, dtype=torch.int64, device=out_on, pin_memory=pin)
    trip = torch.zeros((max(cap, 1), 3), dtype=torch.int32, device=out_on, pin_memory=pin)
    o = lib.jpsi_outputs()
    o.accept_bits, o.track_counts, o.trip_off = acc.data_ptr(), tc.data_ptr(), toff.data_ptr()
    o.triplets, o.trip_capacity = trip.data_ptr(), max(cap, 1)
    torch.cuda.synchronize()
    s, t = lib.jpsi_serve_submit(ctx.ctx, hb, o)
    assert s == 0
    ws, rs, _ = lib.jpsi_serve_wait(ctx.ctx, t, 60000)
    assert ws == 0 and rs == 0 and o.trip_needed == cap
    assert np.array_equal(acc.cpu().numpy().view(np.uint32), ref["accept_bits"])
    assert np.array_equal(tc.cpu().numpy(), ref["track_counts"])
    assert np.array_equal(toff.cpu().numpy(), ref["trip_off"])
    assert np.array_equal(sorted_triplets(toff.cpu().numpy(), trip.cpu().numpy()[:cap], nu),
                          sorted_triplets(ref["trip_off"], ref["triplets"], nu))
    assert lib.jpsi_serve_stop(ctx.ctx) == 0
