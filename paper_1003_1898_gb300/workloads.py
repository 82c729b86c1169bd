"""Seeded synthetic workloads (shapes, seeds, lengths, arrival times).

The benchmark and the tests draw their inputs here.  Only workload
structure lives in this module -- drawn with numpy's PCG64 -- never any of
the generators' arithmetic.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x5EED            # stream i of a handle is seeded from splitmix64(0x5EED + i)
GENS = ("ggl", "xor128", "ranecu", "ranmar", "ranlux", "mt19937")
LUXURY_LEVELS = (24, 48, 97, 223, 389)
PLANAR_LEVELS = (120, 240, 408)     # Section 3.6 planar scheme (its p = 48 is standard too)

# Bulk fills (streams x draws per stream).
SMALL = dict(n_streams=256, n_per=4096)                 # every element checked
ROOFLINE = dict(n_streams=131072, n_per=8192)           # 2^30 draws per dtype
ROOFLINE_MT = dict(n_streams=8192, n_per=131072)        # MT19937: 624-word tables
LUX_SWEEP = dict(n_streams=65536, n_per=4096)           # 2^28 draws per luxury level
JUMP = dict(n=2**30, n_chunks=65536)                    # single sequence from x0 = 1
JUMP_X0 = {"ggl": 1, "ranecu": 1 | (1 << 32),          # RANECU: s1 = s2 = 1
           "xor128": SEED_BASE,                          # XOR128: seeding value s = x0
           "mt19937": 5489}                              # MT19937: init_genrand(5489)

# Batched requests: draws per stream a request is split into.
DRAWS_PER_STREAM = {"mt19937": 65536, "ranmar": 16384}
DEFAULT_DRAWS_PER_STREAM = 4096
BATCH_RANLUX_P = 223


def request_split(gen: str, n: int):
    """Streams and draws per stream of a request for n numbers: ceil(n /
    C_g) streams would take ceil(n / S) draws each; that count is rounded up
    to a multiple of 4 (so that every stream's row starts on a 16-byte
    boundary and the kernels keep their vector stores) and S = ceil(n /
    draws) streams are used.  The first n of the stream-major block are the
    request's output."""
    c = DRAWS_PER_STREAM.get(gen, DEFAULT_DRAWS_PER_STREAM)
    s = -(-n // c)
    per = 4 * -(-(-(-n // s)) // 4)
    return -(-n // per), per


def batched_requests(n_requests: int = 20000, seed: int = 0xB47C, min_len: int = 100,
                     max_len: int = 10**7):
    """Requests with lengths log-uniform in [min_len, max_len], generator
    uniform over the six (RANLUX at p = 223), dtype uint32 or float32 with
    probability 1/2.  Request r's streams are seeded from base seed
    seed + r * 2^32 (disjoint ranges, so no two requests share a stream)."""
    rng = np.random.default_rng(seed)
    lengths = np.floor(10.0 ** rng.uniform(np.log10(min_len), np.log10(max_len),
                                           size=n_requests)).astype(np.int64)
    gens = rng.integers(0, len(GENS), size=n_requests)
    f32 = rng.integers(0, 2, size=n_requests)
    out = []
    for r in range(n_requests):
        g = GENS[int(gens[r])]
        n = int(lengths[r])
        s, per = request_split(g, n)
        out.append({"gen": g, "luxury": BATCH_RANLUX_P if g == "ranlux" else 0, "n": n,
                    "n_streams": s, "n_per": per, "f32": bool(f32[r]),
                    "seed": seed + (r << 32)})
    return out


SERVE_CLIENTS = 512
SERVE_STREAMS = 4096          # divides L*L/2 for every Ising size below
SERVE_ISING_L = (256, 1024, 4096)
SERVE_SWEEPS = 16
SERVE_MEM_CAP = 40e9


def serving_clients(n_clients: int = SERVE_CLIENTS, seed: int = 0x5E5E):
    """(generator, luxury, base seed) per client: half RANLUX p = 223, the
    rest uniform over the other five.  Client c's streams are seeded from
    base seed seed + c * 2^32."""
    rng = np.random.default_rng(seed)
    others = [g for g in GENS if g != "ranlux"]
    out = []
    for c in range(n_clients):
        if c % 2 == 0:
            g, lux = "ranlux", 223
        else:
            g, lux = others[int(rng.integers(0, len(others)))], 0
        out.append((g, lux, seed + (c << 32)))
    return out


def serving_requests(n_requests: int, rate: float, n_clients: int = SERVE_CLIENTS,
                     seed: int = 0xA771, fill_min: int = 10**3, fill_max: int = 10**6,
                     ising_sizes=SERVE_ISING_L, sweeps: int = SERVE_SWEEPS):
    """Poisson arrivals at `rate` per second; each request goes to a client
    uniformly at random and is a fill (log-uniform length in [fill_min,
    fill_max], dtype at random) or an Ising run (L uniform over
    ising_sizes) with probability 1/2 each.  Returns dicts."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    clients = rng.integers(0, n_clients, size=n_requests)
    kinds = rng.integers(0, 2, size=n_requests)
    lens = np.floor(10.0 ** rng.uniform(np.log10(fill_min), np.log10(fill_max), size=n_requests))
    f32 = rng.integers(0, 2, size=n_requests)
    sizes = rng.integers(0, len(ising_sizes), size=n_requests)
    out = []
    for i in range(n_requests):
        if kinds[i] == 0:
            out.append({"rid": i, "client": int(clients[i]), "kind": "fill", "arrival": float(t[i]),
                        "n": int(lens[i]), "f32": bool(f32[i])})
        else:
            out.append({"rid": i, "client": int(clients[i]), "kind": "ising", "arrival": float(t[i]),
                        "L": int(ising_sizes[int(sizes[i])]), "sweeps": sweeps})
    return out


def sample_rows(n_rows: int, k: int, seed: int = 1234) -> np.ndarray:
    """k distinct sorted rows, always including the first and the last."""
    rng = np.random.default_rng(seed)
    k = min(k, n_rows)
    rows = set([0, n_rows - 1])
    while len(rows) < k:
        rows.add(int(rng.integers(0, n_rows)))
    return np.array(sorted(rows), dtype=np.int64)


def jump_offsets(n: int, n_chunks: int, k: int = 4096, seed: int = 4321) -> np.ndarray:
    """Sorted offsets into a jump fill: 0, n-1, 9999, every 16th chunk
    boundary and the draw before it, the rest uniform."""
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
