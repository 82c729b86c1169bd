"""Time one batched Ising half-sweep launch (CUDA events), for tuning and
profiler captures of the half-sweep kernel.

    python -m paper_1003_1898_gb300.isingbench L N_LATTICES [--reps R] [--timed K]

N_LATTICES cold-start lattices of side L with random draws, colour 0, the
critical beta's thresholds.  Prints one line per timed launch: milliseconds
and site updates per second.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import ISING_REQ_DTYPE, prng_ising_half_sweep, prng_ising_thresholds


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("L", type=int)
    ap.add_argument("n_lattices", type=int)
    ap.add_argument("--reps", type=int, default=3, help="untimed launches before the timed ones")
    ap.add_argument("--timed", type=int, default=1, help="timed launches")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    t4, t8 = prng_ising_thresholds(0.4406868)
    g = torch.Generator(device="cuda").manual_seed(1)
    lat = [torch.ones((a.L, a.L), dtype=torch.int8, device="cuda") for _ in range(a.n_lattices)]
    draws = [torch.randint(-2**31, 2**31 - 1, (a.L * a.L // 2,), dtype=torch.int32, device="cuda",
                           generator=g) for _ in range(a.n_lattices)]
    # descriptor rows built once, in the library's struct layout, so a timed
    # launch carries no per-lattice host work
    reqs = np.zeros(a.n_lattices, ISING_REQ_DTYPE)
    for i, (s, d) in enumerate(zip(lat, draws)):
        reqs[i] = (s.data_ptr(), d.data_ptr(), a.L, 0, 8, t4, t8, 0, 0)
    for _ in range(a.reps):
        prng_ising_half_sweep(reqs)
    torch.cuda.synchronize()
    sites = a.n_lattices * a.L * a.L // 2
    for _ in range(a.timed):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        prng_ising_half_sweep(reqs)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(f"ising half-sweep {a.n_lattices} x L={a.L}: {ms:.4f} ms  "
              f"{sites / ms / 1e6:.1f} G site updates/s")


if __name__ == "__main__":
    main()
