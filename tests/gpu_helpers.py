"""Shared pieces of the GPU tests: run the library on a host batch through the
C-ABI binding and compare with the oracle element by element."""
import numpy as np

from helpers import sorted_triplets


def to_device(batch):
    import torch
    d = {k: torch.from_numpy(np.ascontiguousarray(batch[k])).cuda() for k in ("x", "y", "z", "offsets")}
    d["n_events"] = int(batch["n_events"])
    return d


def gpu_select(ctx, batch, form="batched", triplets=True, capacity=None):
    import torch
    d = to_device(batch)
    r = ctx.select(d["x"], d["y"], d["z"], d["offsets"], d["n_events"], triplets=triplets, capacity=capacity,
                   form=form)
    torch.cuda.synchronize()
    out = {"status": r["status"], "trip_needed": r["trip_needed"],
           "accept_bits": r["accept_bits"].cpu().numpy().view(np.uint32),
           "track_counts": r["track_counts"].cpu().numpy(),
           "trip_off": r["trip_off"].cpu().numpy(),
           "triplets": None if r["triplets"] is None else r["triplets"].cpu().numpy()}
    return out


def assert_same(gpu, ref, n_units, check_triplets=True, label=""):
    """Bit-exact: accept bits, track counts, per-unit offsets, and the sorted
    triplet set of every unit."""
    n_events = len(ref["track_counts"])
    assert gpu["status"] == 0, label
    assert gpu["trip_needed"] == ref["trip_needed"], label
    assert np.array_equal(gpu["track_counts"], ref["track_counts"]), (
        label, np.nonzero(gpu["track_counts"] != ref["track_counts"])[0][:10])
    assert np.array_equal(gpu["accept_bits"][: (n_events + 31) // 32], ref["accept_bits"]), label
    assert np.array_equal(gpu["trip_off"], ref["trip_off"]), (
        label, np.nonzero(np.diff(gpu["trip_off"]) != np.diff(ref["trip_off"]))[0][:10])
    if check_triplets:
        a = sorted_triplets(gpu["trip_off"], gpu["triplets"], n_units)
        b = sorted_triplets(ref["trip_off"], ref["triplets"], n_units)
        assert np.array_equal(a, b), label


def gpu_select_stream(ctx, ts, bounds=None, dt=None, form="batched", triplets=True, capacity=None, z_layer=None):
    """The free-streaming selection of a host timeslice (dict of numpy arrays)
    through jpsi_run_stream / jpsi_run_stream_plain; outputs on the host."""
    import torch
    d = {k: torch.from_numpy(np.ascontiguousarray(ts[k])).cuda() for k in ("x", "y", "t", "offsets")}
    z = None if z_layer is not None else torch.from_numpy(np.ascontiguousarray(ts["z"])).cuda()
    zl = None if z_layer is None else torch.from_numpy(np.asarray(z_layer, np.float32)).cuda()
    b = np.asarray(ts["bounds"] if bounds is None else bounds, np.float32)
    db = torch.from_numpy(b.copy()).cuda()
    r = ctx.select_stream(d["x"], d["y"], z, d["t"], d["offsets"], db, ts["dt"] if dt is None else dt,
                          triplets=triplets, capacity=capacity, form=form, z_layer=zl)
    torch.cuda.synchronize()
    return {"status": r["status"], "trip_needed": r["trip_needed"], "error": r.get("error", ""),
            "accept_bits": r["accept_bits"].cpu().numpy().view(np.uint32),
            "track_counts": r["track_counts"].cpu().numpy(),
            "trip_off": r["trip_off"].cpu().numpy(),
            "triplets": None if r["triplets"] is None else r["triplets"].cpu().numpy()}
