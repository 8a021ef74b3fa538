"""Tile-shape autotuner for the fused step kernel.

For a given ensemble, every tile shape compiled into the library for its
lattice is timed on the device (CUDA events around a plain run of step
launches, after a warm-up) through the public API, and the fastest shape is
returned.  Results are cached in a JSON file keyed by lattice, coupling,
precision and the multiset of system sizes, so a later run of the same
ensemble picks its tile without re-timing.
"""
import json
import os

from . import Ensemble, LBError, LB_ERR_UNSUPPORTED

# Compiled variants (must match the tables in csrc/lattice_d2q9.cu and lattice_d3q19.cu):
# D2Q9 tiles are (x, y, 1); D3Q19 tiles are (x, y, z-chunk) of the z-marching kernel;
# the last entry is the resident-CTA target of the register budget (0 = default).
TILES = {
    "D2Q9": [(32, 8, 1, 0), (64, 4, 1, 0), (128, 2, 1, 0)],
    "D3Q19": [(16, 16, 16, 4), (16, 16, 32, 4), (16, 16, 8, 4), (32, 16, 16, 2), (16, 8, 16, 6), (32, 8, 16, 4)],
}
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "lbfluct_tiles.json")


def ensemble_key(systems, precision):
    sizes = sorted((s["nx"], s["ny"], s["nz"]) for s in systems)
    counts = {}
    for sz in sizes:
        counts[sz] = counts.get(sz, 0) + 1
    return "%s/%s/%s/%s" % (systems[0]["lattice"], systems[0]["coupling"], precision,
                            ";".join("%dx%dx%d*%d" % (k + (v,)) for k, v in sorted(counts.items())))


def time_tile(systems, precision, tile, steps=20, warmup=5):
    """Mean milliseconds per step of the step kernel for one tile shape."""
    import torch
    ens = Ensemble(systems, precision=precision, tile=tile[:3], occupancy=tile[3])
    try:
        ens.init(amplitude=0.01)
        ens.step(warmup)
        ens.sync()
        stream = ens.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ens.step(steps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps
    finally:
        ens.close()


def tune(systems, precision="fp32", cache=DEFAULT_CACHE, steps=20, warmup=5, refresh=False):
    """Return (best tile, {tile: ms}) for this ensemble, using the cache when present."""
    key = ensemble_key(systems, precision)
    table = {}
    if cache and os.path.exists(cache) and not refresh:
        try:
            with open(cache) as fh:
                table = json.load(fh)
        except (OSError, ValueError):
            table = {}
        if key in table:
            ent = table[key]
            return tuple(ent["best"]), {tuple(map(int, k.split("x"))): v for k, v in ent["ms"].items()}
    results = {}
    for tile in TILES[systems[0]["lattice"]]:
        try:
            results[tile] = time_tile(systems, precision, tile, steps, warmup)
        except LBError as e:
            if e.status != LB_ERR_UNSUPPORTED:
                raise
    best = min(results, key=results.get)
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        table[key] = {"best": list(best), "ms": {"x".join(map(str, t)): v for t, v in results.items()}}
        with open(cache, "w") as fh:
            json.dump(table, fh, indent=1)
    return best, results
