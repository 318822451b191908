"""Writes the stored expected values under tests/golden/.

Inputs come from the seeded generator (``synth``) and every expected value
from the oracle (``oracle``) alone; nothing here touches the GPU library.
Run from the repository root:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def main():
    gen = {}
    for name, n in (("poisson20_1k", 1000), ("poisson100_1m", 300), ("lognormal_timeslices", 300),
                    ("poisson1500_6st", 2)):
        b = synth.generate(name, 0, n)
        gen[name] = {"n_events": n, "n_hits": int(b["n_hits"]), "sha256": synth.checksum(b)}
    with open(os.path.join(HERE, "synth_checksums.json"), "w") as f:
        json.dump({"note": "sha256 over offsets, x, y, z bytes of events [0, n_events) of each workload; "
                           "written by tests/golden/make_golden.py", "workloads": gen}, f, indent=1)

    b = synth.generate("poisson20_1k")
    res = {}
    for mode_name, mode in (("paper", oracle.MODE_PAPER), ("chain", oracle.MODE_CHAIN)):
        for label, t_xz, t_yz in (("window_0p5", 0.25, 0.25), ("paper_cuts", 0.03, 0.025)):
            p = oracle.params(4, mode, t_xz=t_xz, t_yz=t_yz)
            r = oracle.run(p, b, n_threads=4)
            res[f"{mode_name}_{label}"] = {
                "t_xz": t_xz, "t_yz": t_yz,
                "trip_needed": int(r["trip_needed"]),
                "accepted": int(np.unpackbits(r["accept_bits"].view(np.uint8)).sum()),
                "track_count_sum": int(r["track_counts"].sum()),
                "sha256_triplets_trip_off_track_counts_accept": sha(r["triplets"], r["trip_off"], r["track_counts"],
                                                                    r["accept_bits"]),
            }
    with open(os.path.join(HERE, "oracle_poisson20_1k.json"), "w") as f:
        json.dump({"note": "oracle results on workload poisson20_1k (1000 events, 4 stations); "
                           "written by tests/golden/make_golden.py from oracle/ only", "results": res}, f, indent=1)


if __name__ == "__main__":
    main()
