"""Step-kernel variant autotuner.

For a given ensemble, every step-kernel variant compiled into the library for
its lattice (tile shape, register budget, producer warps; listed by
``lb_kernel_variants``) is timed on the device (CUDA events around a plain run
of step launches, after a warm-up) through the public API, and the fastest is
returned.  Results are cached in a JSON file keyed by lattice, coupling,
precision and the multiset of system sizes, so a later run of the same ensemble
picks its variant without re-timing.  A variant is named by its row
``(x, y, z, occupancy, producer warps, staging, sites per thread)``; ``Ensemble(..., variant=variant_index(...))``
selects it.
"""
import json
import os

from . import Ensemble, LBError, LB_ERR_UNSUPPORTED, kernel_variants

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "lbfluct_tiles.json")


def variants(lattice):
    """The compiled variants of a lattice, row 0 the default."""
    return kernel_variants(lattice)


def variant_index(lattice, row):
    """The ``variant`` option (1-based) that selects a compiled variant row."""
    return variants(lattice).index(tuple(row)) + 1


def ensemble_key(systems, precision):
    sizes = sorted((s["nx"], s["ny"], s["nz"]) for s in systems)
    counts = {}
    for sz in sizes:
        counts[sz] = counts.get(sz, 0) + 1
    return "%s/%s/%s/%s" % (systems[0]["lattice"], systems[0]["coupling"], precision,
                            ";".join("%dx%dx%d*%d" % (k + (v,)) for k, v in sorted(counts.items())))


def time_variant(systems, precision, index, steps=20, warmup=5):
    """Mean milliseconds per step with compiled variant ``index`` (0-based)."""
    import torch
    ens = Ensemble(systems, precision=precision, variant=index + 1)
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
    """Return (best variant row, {row: ms}) for this ensemble, using the cache when present."""
    lattice = systems[0]["lattice"]
    rows = variants(lattice)
    key = ensemble_key(systems, precision)
    table = {}
    if cache and os.path.exists(cache) and not refresh:
        try:
            with open(cache) as fh:
                table = json.load(fh)
        except (OSError, ValueError):
            table = {}
        ent = table.get(key)
        if ent is not None and tuple(ent["best"]) in rows:
            return tuple(ent["best"]), {tuple(map(int, k.split("x"))): v for k, v in ent["ms"].items()}
    results = {}
    for i, row in enumerate(rows):
        try:
            results[row] = time_variant(systems, precision, i, steps, warmup)
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
