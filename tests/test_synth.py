"""The seeded input generator: determinism, sub-range generation and the
shapes the workloads are meant to have."""
import json
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _xoshiro_ref(s, n):
    """xoshiro256** written out from its published definition (Blackman-Vigna)."""
    M = (1 << 64) - 1
    s = list(s)
    out = []
    rotl = lambda x, k: ((x << k) | (x >> (64 - k))) & M  # noqa: E731
    for _ in range(n):
        out.append((rotl((s[1] * 5) & M, 7) * 9) & M)
        t = (s[1] << 17) & M
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = rotl(s[3], 45)
    return out


def test_xoshiro_and_splitmix(synth_mod):
    import ctypes
    lib = synth_mod._load()
    seeds = (0x0123456789ABCDEF, 0xFEDCBA9876543210, 1, 0xDEADBEEF)
    out = (ctypes.c_uint64 * 16)()
    lib.jpsi_synth_xoshiro_first(*seeds, 16, out)
    assert list(out) == _xoshiro_ref(seeds, 16)
    # SplitMix64 finaliser of 0x9e3779b97f4a7c15 (first output for seed 0)
    assert lib.jpsi_synth_splitmix_mix(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF


def test_log_exp_series_accuracy(synth_mod):
    lib = synth_mod._load()
    for v in np.geomspace(1e-300, 1e300, 500):
        assert abs(lib.jpsi_synth_log(v) - math.log(v)) <= 4e-16 * max(1.0, abs(math.log(v)))
    for v in np.linspace(-700, 700, 500):
        assert abs(lib.jpsi_synth_exp(v) / math.exp(v) - 1.0) <= 1e-13


def test_checksums_golden(synth_mod):
    with open(os.path.join(HERE, "golden", "synth_checksums.json")) as f:
        gold = json.load(f)["workloads"]
    for name, g in gold.items():
        b = synth_mod.generate(name, 0, g["n_events"])
        assert b["n_hits"] == g["n_hits"]
        assert synth_mod.checksum(b) == g["sha256"], name


def test_subrange_and_threads(synth_mod):
    full = synth_mod.generate("poisson100_1m", 0, 200, n_threads=1)
    part = synth_mod.generate("poisson100_1m", 150, 30, n_threads=3)
    o = full["offsets"]
    S3 = 12
    a, b = o[150 * S3], o[180 * S3]
    for k in ("x", "y", "z"):
        assert np.array_equal(part[k], full[k][a:b])
    assert np.array_equal(part["offsets"], o[150 * S3:180 * S3 + 1] - a)


def test_workload_shapes(synth_mod):
    b = synth_mod.generate("poisson20_1k", truth=True)
    counts = np.diff(b["offsets"]).reshape(1000, 12)
    n_mu = (b["truth"] > 0).reshape(-1)
    # Poisson(20) background + muons; ~30 % of events with two muons
    assert abs(counts.mean() - (20 + 0.6)) < 0.3
    ev_mu = np.add.reduceat(n_mu.astype(int), b["offsets"][:-1:12]) // 12
    assert 0.26 < np.mean(ev_mu == 2) < 0.34
    # layer z = station z +- 10 cm
    zl = np.repeat(np.tile([120, 130, 140, 155, 165, 175, 190, 200, 210, 225, 235, 245], 1000), counts.reshape(-1))
    assert np.array_equal(b["z"], zl.astype(np.float32))
    # background in the annulus 15 < r < 0.4 z
    bg = b["truth"] == 0
    r = np.hypot(b["x"][bg], b["y"][bg])
    assert r.min() >= 15.0 - 1e-4 and np.all(r <= 0.4 * b["z"][bg] + 1e-4)
    # muon hits within 5 sigma of a straight line from the target
    mu = ~bg
    assert np.all(np.abs(b["x"][mu]) <= 0.35 * b["z"][mu] + 0.5)


def test_inverse_r2_density(synth_mod):
    b = synth_mod.generate("poisson100_1m", 0, 300, truth=True)
    bg = b["truth"] == 0
    r = np.hypot(b["x"][bg], b["y"][bg]) / 15.0
    R = 0.4 * b["z"][bg] / 15.0
    u = np.log(r) / np.log(R)  # uniform in [0, 1) for an area density ~ 1/r^2
    assert abs(u.mean() - 0.5) < 0.01 and abs(np.mean(u < 0.25) - 0.25) < 0.01
    counts = np.diff(b["offsets"])
    assert abs(counts.mean() - 100.18) < 1.0


def test_lognormal_multiplicity(synth_mod):
    w = synth_mod.WORKLOADS["lognormal_timeslices"]
    c = synth_mod.layer_counts(w, 0, 20000).astype(np.float64)
    lam = c.mean(axis=1)
    assert c.min() >= 5 and c.max() <= 1500 + 2
    assert 50 < np.median(lam) < 72
    sizes = synth_mod.timeslice_sizes(w)
    assert len(sizes) == 64 and sizes.min() >= 10_000 and sizes.max() <= 100_000
