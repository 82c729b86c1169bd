"""Autotuner for the fill kernels' launch tiles.

For each generator (RANLUX: each luxury p) it times one fill of a given
workload shape with every tile compiled into the library (threads per CTA,
staged draws per thread, staging buffers), keeps the fastest, and can save
the choice as JSON so later processes apply it with ``apply()`` before
filling.  Timing uses CUDA events on the current stream after a warm-up
fill; outputs larger than L2 are used so no flush is needed.

  python -m paper_1003_1898_gb300.tune [--out tuned_tiles.json]
"""
from __future__ import annotations

import argparse
import json
import os

from . import GEN_NAMES, LUXURY_P, PLANAR_P, prng_create, prng_destroy, prng_fill_f32, prng_fill_u32, \
    prng_get_tile, prng_set_tile

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuned_tiles.json")

TILES = {
    "simple": [(128, 32, 1), (128, 32, 2), (128, 64, 1), (256, 32, 1)],
    "ggl": [(128, 128, 1), (256, 128, 1), (128, 32, 1), (128, 64, 1)],
    "ranecu": [(128, 128, 1), (256, 128, 1), (128, 32, 1), (128, 64, 1)],
    # cols = 56: a per-row ring written out 32 words at a time by each warp
    "ranlux": [(64, 48, 1), (128, 48, 1), (256, 48, 1), (64, 56, 1), (128, 56, 1), (256, 56, 1)],
    "ranlux_high": [(64, 48, 1), (128, 48, 1), (256, 48, 1), (64, 96, 1),   # p >= 97
                    (64, 56, 1), (128, 56, 1)],
    "ranmar": [(128, 128, 1), (256, 128, 1)],
    "mt19937": [(64, 624, 1), (128, 624, 1), (256, 624, 1), (32, 624, 2), (64, 624, 2),
                (128, 624, 2), (256, 624, 2)],
}

# Workload shapes the tiles are tuned for: the roofline bulk fill, and for
# RANLUX at p >= 97 (not part of that fill) the luxury sweep.
SHAPES = {"mt19937": (8192, 131072)}
DEFAULT_SHAPE = (131072, 8192)
LUXURY_SHAPE = (65536, 4096)


def tiles_for(gen: str, luxury: int = 0):
    """Tiles compiled for a generator (RANLUX at p >= 97 has one more)."""
    if gen == "ranlux" and luxury >= 97:
        return TILES["ranlux_high"]
    return TILES.get(gen, TILES["simple"])


def key(gen: str, luxury: int = 0) -> str:
    return f"ranlux_p{luxury}" if gen == "ranlux" else gen


def time_fill(gen: str, tile, n_streams: int, n_per: int, luxury: int = 0, dtype: str = "u32",
              reps: int = 5) -> float:
    """Median milliseconds of one fill with the given tile."""
    import torch
    prng_set_tile(gen, luxury, *tile)
    h = prng_create(gen, 0x5EED, n_streams, luxury)
    try:
        tdt = torch.float32 if dtype == "f32" else torch.int32
        out = torch.empty(n_streams * n_per, dtype=tdt, device="cuda")
        fill = prng_fill_f32 if dtype == "f32" else prng_fill_u32
        fill(h, out, n_per)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fill(h, out, n_per)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        del out
    finally:
        prng_destroy(h)
    ts.sort()
    return ts[len(ts) // 2]


def tune(gens=GEN_NAMES, luxuries=LUXURY_P + PLANAR_P[1:], reps: int = 5, verbose: bool = True) -> dict:
    """Time every compiled tile and return {key: {"tile": [...], "ms": {...}}};
    a tile's ms is the sum of one u32 and one f32 fill of the shape."""
    result = {}
    jobs = []
    for g in gens:
        if g == "ranlux":
            jobs += [(g, p) for p in luxuries]
        else:
            jobs.append((g, 0))
    for g, lux in jobs:
        ns, nper = LUXURY_SHAPE if (g == "ranlux" and lux >= 97) else SHAPES.get(g, DEFAULT_SHAPE)
        before = prng_get_tile(g, lux)
        ms = {}
        for t in tiles_for(g, lux):   # a u32 fill plus an f32 fill, as the benchmark step does
            ms[",".join(map(str, t))] = (time_fill(g, t, ns, nper, lux, "u32", reps=reps) +
                                         time_fill(g, t, ns, nper, lux, "f32", reps=reps))
        best = min(ms, key=ms.get)
        tile = [int(x) for x in best.split(",")]
        prng_set_tile(g, lux, *tile)
        result[key(g, lux)] = {"tile": tile, "ms": ms, "shape": [ns, nper],
                               "before": list(before)}
        if verbose:
            print(f"{key(g, lux):12s} best {tile}  " +
                  "  ".join(f"{k}:{v:.3f}" for k, v in ms.items()), flush=True)
    return result


def apply(cache: dict):
    for k, v in cache.items():
        if k.startswith("ranlux_p"):
            prng_set_tile("ranlux", int(k[len("ranlux_p"):]), *v["tile"])
        elif k in GEN_NAMES:
            prng_set_tile(k, 0, *v["tile"])


def load(path: str = DEFAULT_CACHE) -> dict | None:
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def load_and_apply(path: str = DEFAULT_CACHE) -> bool:
    c = load(path)
    if c is None:
        return False
    apply(c)
    return True


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_CACHE)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    from . import build
    build.build()
    res = tune(reps=args.reps)
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
    print(args.out)


if __name__ == "__main__":
    main()
