"""The allocation-free counting entry point (jpsi_select_noalloc) against the
regular one (jpsi_run).

It exists for callers that must not allocate device memory while they run
(pre-reserved memory for a latency budget, memory owned by a host program's
allocator).  Its scratch is a fixed array inside the library; these checks
call it twice in a row, so the second call also shows that what the first
left in that array does not leak into the result.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1810_11966_gb300 as jp
    jp.load(build_if_missing=True)
    return jp


def _regular(lib, p, d, n):
    import torch
    ctx = lib.Context(p)
    r = ctx.select(d["x"], d["y"], d["z"], d["offsets"], n, triplets=False)
    torch.cuda.synchronize()
    assert r["status"] == 0
    tc = r["track_counts"].cpu().numpy()
    uc = np.diff(r["trip_off"].cpu().numpy())
    ctx.close()
    return tc, uc


@pytest.mark.parametrize("mode", [0, 1])
def test_noalloc_matches_regular_entry_point(lib, synth_mod, mode):
    import torch
    S = 4
    n = 20000
    b = synth_mod.generate("poisson100_1m", 0, n)
    d = {k: torch.from_numpy(b[k]).cuda() for k in ("x", "y", "z", "offsets")}
    p = lib.params(S, mode, t_xz=0.25)
    tc_ref, uc_ref = _regular(lib, p, d, n)
    batch = lib.make_batch(d["x"], d["y"], d["z"], d["offsets"], n, b["n_hits"])
    st = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row share the library's scratch array
        tc = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        uc = torch.full((n * S,), -7, dtype=torch.int32, device="cuda")
        s = lib.jpsi_select_noalloc(p, batch, tc.data_ptr(), uc.data_ptr(), st)
        assert s == lib.JPSI_OK, lib.jpsi_strerror(s)
        torch.cuda.synchronize()
        assert np.array_equal(tc.cpu().numpy(), tc_ref)
        assert np.array_equal(uc.cpu().numpy(), uc_ref)


def test_noalloc_rejects_batches_beyond_its_limits(lib, synth_mod):
    import torch
    p = lib.params(4, 1, t_xz=0.25)
    # the hit-disjoint accept rule changes accept bits only, which this entry
    # point does not return: refused
    nb = lib.jpsi_batch()
    assert lib.jpsi_select_noalloc(lib.params(4, 1, t_xz=0.25, distinct_hits=1), nb, None, None, 0) == lib.JPSI_EINVAL
    # more events than the fixed scratch holds: refused before anything runs
    big = lib.jpsi_batch()
    big.n_events, big.n_hits = (1 << 18) + 1, 0
    big.offsets = ctypes.c_void_p(1)
    assert lib.jpsi_select_noalloc(p, big, None, None, 0) == lib.JPSI_EINVAL
    # an event larger than a warp tile needs the other kernels: refused
    b = synth_mod.generate("lognormal_timeslices", 0, 400)
    assert np.diff(b["offsets"]).max() > 192
    d = {k: torch.from_numpy(b[k]).cuda() for k in ("x", "y", "z", "offsets")}
    tc = torch.empty(400, dtype=torch.int32, device="cuda")
    uc = torch.empty(1600, dtype=torch.int32, device="cuda")
    batch = lib.make_batch(d["x"], d["y"], d["z"], d["offsets"], 400, b["n_hits"])
    st = torch.cuda.current_stream().cuda_stream
    assert lib.jpsi_select_noalloc(p, batch, tc.data_ptr(), uc.data_ptr(), st) == lib.JPSI_EINVAL
    # and the entry point still works afterwards
    b = synth_mod.generate("poisson20_1k", 0, 500)
    d = {k: torch.from_numpy(b[k]).cuda() for k in ("x", "y", "z", "offsets")}
    tc = torch.empty(500, dtype=torch.int32, device="cuda")
    uc = torch.empty(2000, dtype=torch.int32, device="cuda")
    batch = lib.make_batch(d["x"], d["y"], d["z"], d["offsets"], 500, b["n_hits"])
    assert lib.jpsi_select_noalloc(p, batch, tc.data_ptr(), uc.data_ptr(), st) == lib.JPSI_OK
    tc_ref, uc_ref = _regular(lib, p, d, 500)
    assert np.array_equal(tc.cpu().numpy(), tc_ref) and np.array_equal(uc.cpu().numpy(), uc_ref)
