"""The oracle against its stored results on the small workload (written by
tests/golden/make_golden.py from the oracle alone).  A change to the oracle's
arithmetic shows up here and must cite the paper passage that justifies it."""
import hashlib
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_golden(oracle_mod, synth_mod):
    with open(os.path.join(HERE, "golden", "oracle_poisson20_1k.json")) as f:
        gold = json.load(f)["results"]
    b = synth_mod.generate("poisson20_1k")
    for key, g in gold.items():
        mode = oracle_mod.MODE_PAPER if key.startswith("paper_") else oracle_mod.MODE_CHAIN
        r = oracle_mod.run(oracle_mod.params(4, mode, t_xz=g["t_xz"], t_yz=g["t_yz"]), b, n_threads=2)
        h = hashlib.sha256()
        for a in (r["triplets"], r["trip_off"], r["track_counts"], r["accept_bits"]):
            h.update(np.ascontiguousarray(a).tobytes())
        assert r["trip_needed"] == g["trip_needed"], key
        assert int(r["track_counts"].sum()) == g["track_count_sum"], key
        assert h.hexdigest() == g["sha256_triplets_trip_off_track_counts_accept"], key
