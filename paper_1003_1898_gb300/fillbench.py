"""Time one generator fill in isolation (CUDA events), for tile studies and
profiler captures of a single kernel.

    python -m paper_1003_1898_gb300.fillbench GEN {u32,f32} N_STREAMS N_PER
        [--luxury P] [--reps R] [--timed K] [--jump] [--skip] [--tile T,C,S]

--jump times prng_fill_jump_* (GGL or RANECU, N_STREAMS chunks of N_PER
draws); --skip times prng_skip of N_PER draws per stream (no output); f64
fills write N_PER doubles per stream (2 N_PER draws).  The
tiles tuned for this machine (tuned_tiles.json) are applied first, then
--tile (threads, columns, stages) for GEN if given.  Prints
one line per timed call: milliseconds, numbers/s and written GB/s.
"""
from __future__ import annotations

import argparse

import torch

from . import (GEN_IDS, prng_create, prng_destroy, prng_fill_f32, prng_fill_f64, prng_fill_jump_f32,
               prng_fill_jump_u32, prng_fill_u32, prng_set_tile, prng_skip)
from . import tune
from .workloads import JUMP_X0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("gen", choices=sorted(GEN_IDS))
    ap.add_argument("dtype", choices=["u32", "f32", "f64"])
    ap.add_argument("n_streams", type=int)
    ap.add_argument("n_per", type=int)
    ap.add_argument("--luxury", type=int, default=223)
    ap.add_argument("--reps", type=int, default=3, help="untimed calls before the timed one")
    ap.add_argument("--timed", type=int, default=1, help="timed calls")
    ap.add_argument("--jump", action="store_true")
    ap.add_argument("--skip", action="store_true")
    ap.add_argument("--tile", default=None)
    a = ap.parse_args(argv)
    tune.load_and_apply()
    if a.tile:
        prng_set_tile(a.gen, a.luxury if a.gen == "ranlux" else 0, *map(int, a.tile.split(",")))
    n = a.n_streams * a.n_per
    f32 = a.dtype == "f32"
    tdt = {"f32": torch.float32, "f64": torch.float64}.get(a.dtype, torch.int32)
    out = None if a.skip else torch.empty(n, dtype=tdt, device="cuda")
    h = None
    if a.jump:
        fj = prng_fill_jump_f32 if f32 else prng_fill_jump_u32
        call = lambda: fj(a.gen, JUMP_X0[a.gen], n, a.n_streams, out)
    else:
        h = prng_create(a.gen, 0x5EED, a.n_streams, a.luxury)
        fill = {"f32": prng_fill_f32, "f64": prng_fill_f64}.get(a.dtype, prng_fill_u32)
        call = (lambda: prng_skip(h, a.n_per)) if a.skip else (lambda: fill(h, out, a.n_per))
    for _ in range(a.reps):
        call()
    torch.cuda.synchronize()
    for _ in range(a.timed):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        gbs = 0.0 if a.skip else out.element_size() * n / ms / 1e6
        print(f"{a.gen} {a.dtype} {a.n_streams}x{a.n_per}{' jump' if a.jump else ''}"
              f"{' skip' if a.skip else ''}: {ms:.4f} ms  {n / ms / 1e9:.3f} T/s  {gbs:.0f} GB/s")
    if h is not None:
        prng_destroy(h)


if __name__ == "__main__":
    main()
