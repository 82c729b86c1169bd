"""Seeded synthetic inputs shared by the parity tests and the benchmark.

Only workload shapes, seeds and sampling positions live here (drawn with
numpy's own PCG64); none of the generators' arithmetic does.
"""
import numpy as np

SEED_BASE = 0x5EED            # stream i of a handle is seeded from splitmix64(0x5EED + i)
GENS = ("ggl", "xor128", "ranecu", "ranmar", "ranlux", "mt19937")
LUXURY_LEVELS = (24, 48, 97, 223, 389)

# Bulk-fill workloads (streams x draws per stream).
SMALL = dict(n_streams=256, n_per=4096)                 # every element checked
ROOFLINE = dict(n_streams=131072, n_per=8192)           # 2^30 draws per dtype
ROOFLINE_MT = dict(n_streams=8192, n_per=131072)        # MT19937: 624-word tables
LUX_SWEEP = dict(n_streams=65536, n_per=4096)           # 2^28 draws per luxury level
JUMP = dict(n=2**30, n_chunks=65536)                    # single sequence from x0 = 1
JUMP_X0 = {"ggl": 1, "ranecu": 1 | (1 << 32)}           # RANECU: s1 = s2 = 1


def sample_rows(n_rows: int, k: int, seed: int = 1234) -> np.ndarray:
    """k distinct sorted rows, always including the first and the last."""
    rng = np.random.default_rng(seed)
    k = min(k, n_rows)
    rows = set([0, n_rows - 1])
    while len(rows) < k:
        rows.add(int(rng.integers(0, n_rows)))
    return np.array(sorted(rows), dtype=np.int64)


def jump_offsets(n: int, n_chunks: int, k: int = 4096, seed: int = 4321) -> np.ndarray:
    """k sorted offsets into a jump fill: 0, n-1, every 16th chunk boundary
    (and the draw before it), the rest uniform."""
    L = -(-n // n_chunks)
    rng = np.random.default_rng(seed)
    pts = {0, n - 1}
    if n > 9999:
        pts.add(9999)   # Park-Miller's check value sits at draw 10000 of GGL from x0 = 1
    for c in range(0, n_chunks, 16):
        b = c * L
        if b < n:
            pts.add(b)
            if b > 0:
                pts.add(b - 1)
    while len(pts) < k:
        pts.add(int(rng.integers(0, n)))
    return np.array(sorted(pts), dtype=np.uint64)
