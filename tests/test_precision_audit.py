"""FP64 audit of the FP32 reference arithmetic (the paper fixes no precision).

The oracle evaluates the same fit and cuts in double from the same float
inputs; this counts the triplet, candidate and accept decisions that flip on
samples of every workload.  Flips are only possible for triplets whose
summed squared residual lies within rounding distance of the cut, so they
must be rare; the FP32 result stays the reference.  Sample sizes scale with
JPSI_AUDIT_SCALE (default 1); the printed line is the audit record.
"""
import json
import os

import numpy as np
import pytest

from helpers import sorted_triplets

SCALE = float(os.environ.get("JPSI_AUDIT_SCALE", "1"))

CASES = [
    # workload, events at scale 1, stations, window
    ("poisson20_1k", 1000, 4, 0.5),
    ("poisson100_1m", 6000, 4, 0.5),
    ("lognormal_timeslices", 3000, 4, 0.5),
    ("lognormal_stream", 3000, 4, 0.5),
    ("poisson1500_6st", 8, 6, 1.0),
]


def flips(oracle_mod, b, S, t):
    p = oracle_mod.params(S, oracle_mod.MODE_CHAIN, t_xz=t)
    r32 = oracle_mod.run(p, b, n_threads=os.cpu_count() or 1)
    r64 = oracle_mod.run(p, b, n_threads=os.cpu_count() or 1, fp64=True)
    n_units = b["n_events"] * S
    a = {tuple(v) for v in sorted_triplets(r32["trip_off"], r32["triplets"], n_units)}
    c = {tuple(v) for v in sorted_triplets(r64["trip_off"], r64["triplets"], n_units)}
    return {"events": int(b["n_events"]), "triplets_fp32": len(a), "triplet_flips": len(a ^ c),
            "candidate_flips": int(np.sum(r32["track_counts"] != r64["track_counts"])),
            "accept_flips": int(np.sum(r32["accept_bits"] != r64["accept_bits"]))}


@pytest.mark.parametrize("name,n,S,w", CASES)
def test_fp64_flips_are_rare(oracle_mod, synth_mod, name, n, S, w):
    m = max(1, int(n * SCALE))
    b = synth_mod.generate(name, 0, m)
    f = flips(oracle_mod, b, S, w * w)
    print("AUDIT", json.dumps({"workload": name, **f}))
    # a flip needs S within ~1e-6 relative of the cut: at most a few per 10^4 triplets
    assert f["triplet_flips"] <= max(3, f["triplets_fp32"] // 10000)
    assert f["accept_flips"] <= max(1, m // 10000)
