"""bench.py on the CPU: the reference arm (the oracle on the host cores) runs
without a GPU, its JSON line carries the contract's keys, and under torchrun
with two ranks only rank 0 works and prints; the served-from-device check's
canonical form of triplet rows ignores their order inside a unit; the
roofline arithmetic (algorithmic bytes, issue-slot peak) is the stated one."""
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


def test_roofline_arithmetic():
    # algorithmic bytes: each hit once (x, y, z), the CSR offsets, per-unit and
    # track counts and the class byte; PAPER mode: the trigger station only
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    S, n = 4, 2
    assert bench.algorithmic_bytes(n, 10, S) == 12 * 10 + 4 * (n * 3 * S + 1) + 4 * n * S + 4 * n + n
    # two events, 4 stations x 3 layers; trigger station 3 holds 1 + 2 + 0 and 3 + 0 + 1 hits
    counts = np.zeros((n, S, 3), np.int64)
    counts[0, 3] = (1, 2, 0)
    counts[1, 3] = (3, 0, 1)
    counts[:, :3] = 5
    off = np.concatenate([[0], np.cumsum(counts.ravel())]).astype(np.int32)
    assert bench.algorithmic_bytes(n, int(off[-1]), S, offsets=off, trigger=3) == \
        12 * 7 + 4 * 4 * n + 4 * n * S + 4 * n + n
    r = bench.issue_roofline(1000.0, 2_000_000, 2.0, 152, 2070.0)
    assert r["peak"] == 152 * 4 * 2070e6
    assert abs(r["achieved"] - 1000.0 * 2_000_000 / 0.002) < 1e-3 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert bench.issue_roofline(None, 1, 1.0, 152, 2070.0)["frac"] is None
