"""Batch construction helpers shared by the tests (no selection arithmetic)."""
import numpy as np


def make_batch(events, n_stations):
    """events: list over events of list over (station*3 + layer) of hit lists
    [(x, y, z), ...].  Returns the dict layout the oracle and the library take."""
    xs, ys, zs, off = [], [], [], [0]
    for ev in events:
        assert len(ev) == n_stations * 3
        for layer in ev:
            for (x, y, z) in layer:
                xs.append(x)
                ys.append(y)
                zs.append(z)
            off.append(len(xs))
    return {
        "x": np.array(xs, np.float32),
        "y": np.array(ys, np.float32),
        "z": np.array(zs, np.float32),
        "offsets": np.array(off, np.int32),
        "n_events": len(events),
        "n_hits": len(xs),
        "n_stations": n_stations,
    }


def layer_z(n_stations, station_z=(130.0, 165.0, 200.0, 235.0, 270.0, 305.0), dz=10.0):
    return [station_z[s] + (l - 1) * dz for s in range(n_stations) for l in range(3)]


def line_event(n_stations, tracks, noise=None, rng=None, sigma=0.0, extra_bg=0, bg_radius=(15.0, 0.4)):
    """An event with straight tracks from the target (slopes tx, ty) hitting
    every layer, optional Gaussian smear and uniform background."""
    zl = layer_z(n_stations)
    ev = []
    for li, z in enumerate(zl):
        hits = []
        for (tx, ty) in tracks:
            dx = rng.normal(0, sigma) if (rng is not None and sigma > 0) else 0.0
            dy = rng.normal(0, sigma) if (rng is not None and sigma > 0) else 0.0
            hits.append((tx * z + dx, ty * z + dy, z))
        for _ in range(extra_bg):
            r = rng.uniform(bg_radius[0], bg_radius[1] * z)
            ph = rng.uniform(0, 2 * np.pi)
            hits.append((r * np.cos(ph), r * np.sin(ph), z))
        ev.append(hits)
    return ev


def sorted_triplets(trip_off, triplets, n_units):
    """Per-unit canonical (i, j, k) sort of a CSR triplet list -> [n,4] with unit id."""
    if triplets is None or len(triplets) == 0:
        return np.zeros((0, 4), np.int64)
    unit = np.repeat(np.arange(n_units), np.diff(trip_off))
    a = np.concatenate([unit[:, None], np.asarray(triplets, np.int64).reshape(-1, 3)], axis=1)
    order = np.lexsort((a[:, 3], a[:, 2], a[:, 1], a[:, 0]))
    return a[order]


def accept_list(bits, n_events):
    v = np.unpackbits(np.asarray(bits, np.uint32).view(np.uint8), bitorder="little")
    return v[:n_events].astype(bool)


def shared_hit_event(n_stations, third, dz=10.0, pitch=35.0, z0=120.0):
    """Every station: two close tracks in layers 0 and 2 and one middle-layer
    hit between them, so the trigger station's passing triplets all use that
    hit; `third` adds a separate track through every layer."""
    ev = []
    for s in range(n_stations):
        for l in range(3):
            z = z0 + pitch * s + dz * (l - 1)
            hits = [(0.1 * z + 0.4, 0.1 * z, z)] if l == 1 else [(0.1 * z, 0.1 * z, z), (0.1 * z + 0.8, 0.1 * z, z)]
            if third:
                hits.append((-0.2 * z, 0.15 * z, z))
            ev.append(hits)
    return ev
