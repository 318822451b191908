"""The multi-rank path of bench.py on CPU: two gloo ranks each take their own
event range (no data exchange), synchronise with a barrier, and the job time is
the maximum over ranks.  The oracle stands in for the GPU run here; the
ranks' concatenated results must equal one run over all events."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n_per_rank, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import oracle
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    e0, n = bench.shard(rank, n_per_rank)
    b = synth.generate("poisson20_1k", e0, n)
    dist.barrier()
    r = oracle.run(oracle.params(4, 1, t_xz=0.25), b, n_threads=1)
    job = bench.max_over_ranks(10.0 * (rank + 1), dist)  # slowest rank's time
    np.save(os.path.join(out_dir, f"tc{rank}.npy"), r["track_counts"])
    np.save(os.path.join(out_dir, f"uc{rank}.npy"), r["unit_counts"])
    with open(os.path.join(out_dir, f"job{rank}.txt"), "w") as f:
        f.write(f"{e0} {n} {job}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_events(tmp_path, oracle_mod, synth_mod):
    import torch.multiprocessing as mp
    world, n = 2, 150
    mp.start_processes(_rank_main, args=(world, _free_port(), n, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    jobs = [open(tmp_path / f"job{r}.txt").read().split() for r in range(world)]
    assert [(int(a), int(b)) for a, b, _ in jobs] == [(0, n), (n, n)]      # disjoint, contiguous shards
    assert all(float(j[2]) == 20.0 for j in jobs)                          # max over ranks, on every rank
    tc = np.concatenate([np.load(tmp_path / f"tc{r}.npy") for r in range(world)])
    uc = np.concatenate([np.load(tmp_path / f"uc{r}.npy") for r in range(world)])
    whole = oracle_mod.run(oracle_mod.params(4, 1, t_xz=0.25), synth_mod.generate("poisson20_1k", 0, world * n))
    assert np.array_equal(tc, whole["track_counts"]) and np.array_equal(uc, whole["unit_counts"])


def test_bench_roofline_helpers(monkeypatch, tmp_path):
    """Host arithmetic of the bench's roofline fields."""
    import json as _json
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    r = bench.issue_roofline(10.0, 100, 1.0, 152, 2000.0)
    assert r["peak"] == 152 * 4 * 2000e6
    assert r["achieved"] == 10.0 * 100 / 1e-3 and r["frac"] == r["achieved"] / r["peak"]
    assert bench.issue_roofline(None, 100, 1.0, 152, 2000.0)["frac"] is None
    # a record taken on other kernel sources is not used
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"k": {"w": {"dram_bytes_per_event": 5.0, "inst_per_event": 7.0, "source_hash": bench.kernel_source_hash()}}}
    (prof / "ncu_traffic.json").write_text(_json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["k"]["w"]["source_hash"])
    assert bench.ncu_traffic("k", "w") == 5.0 and bench.ncu_record("k", "w", "inst_per_event") == 7.0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "other")
    assert bench.ncu_traffic("k", "w") is None
    # algorithmic bytes of the counting kernel: hits, offsets, counts, class byte
    assert bench.algorithmic_bytes(2, 10, 4) == 12 * 10 + 4 * (2 * 12 + 1) + 4 * 2 * 4 + 4 * 2 + 2
    # PAPER mode: only the trigger station's hits (station 1: one hit in event 0, none in event 1)
    # and its 4 offsets per event
    off = np.array([0, 1, 1, 2, 3, 3, 3] + [3, 4, 4, 4, 4, 4], np.int32)  # 2 events x 2 stations x 3 layers
    assert bench.algorithmic_bytes(2, 4, 2, offsets=off, trigger=1) == 12 * 1 + 4 * 4 * 2 + 4 * 2 * 2 + 4 * 2 + 2
