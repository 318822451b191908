"""bench.py's reference arm (the oracle on the host cores) runs without a GPU:
its JSON line carries the contract's keys, and under torchrun with two ranks
only rank 0 works and prints."""
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
