"""bench.py on the CPU: the reference arm (the oracle on the host cores) runs
without a GPU, its JSON line carries the contract's keys, and under torchrun
with two ranks only rank 0 works and prints; the served-from-device check's
canonical form of triplet rows ignores their order inside a unit."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_line():
    out = subprocess.check_output([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                   "--ref-events", "300", "--steps", "2", "--warmup", "3"], cwd=ROOT, text=True,
                                  timeout=600)
    (line,) = _lines(out)
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "events/s"
    assert line["steps"] == 2 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "events/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_two_ranks_print_once():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = subprocess.check_output([sys.executable, "-m", "torch.distributed.run", "--nnodes", "1",
                                   "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port", str(port),
                                   os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                                   "--ref-events", "200", "--steps", "1", "--warmup", "3"],
                                  cwd=ROOT, text=True, timeout=600, stderr=subprocess.DEVNULL)
    (line,) = _lines(out)
    assert line["impl"] == "reference" and line["n_gpus"] == 2


def test_canonical_rows_ignore_order_inside_a_unit():
    # the served-from-device check compares triplet rows per unit as sets
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(5)
    counts = np.array([3, 0, 5, 1, 4])
    toff = torch.from_numpy(np.concatenate([[0], np.cumsum(counts)]).astype(np.int64))
    rows = torch.from_numpy(rng.integers(0, 4, size=(int(counts.sum()), 3)).astype(np.int32))
    base = bench.canonical_rows(torch, toff, rows)
    # each unit's rows permuted: the same canonical form
    perm = np.concatenate([o + rng.permutation(c) for o, c in zip(toff[:-1].numpy(), counts)]).astype(np.int64)
    assert torch.equal(bench.canonical_rows(torch, toff, rows[torch.from_numpy(perm)]), base)
    # each unit's rows sorted lexicographically, units in order
    for u, c in enumerate(counts):
        seg = base[int(toff[u]): int(toff[u]) + c].tolist()
        assert seg == sorted(seg) and sorted(seg) == sorted(rows[int(toff[u]): int(toff[u]) + c].tolist())
    # one changed value changes it (the unit boundaries are the offsets,
    # which the check compares on their own)
    changed = rows.clone()
    changed[4, 1] += 1
    assert not torch.equal(bench.canonical_rows(torch, toff, changed), base)
