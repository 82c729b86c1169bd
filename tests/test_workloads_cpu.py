"""Host-side pieces without a GPU: the seeded workloads (request splits,
batched and serving mixes, jump-fill check offsets) and the library's launch
tile table (prng_set_tile / prng_get_tile touch no device)."""
import numpy as np
import pytest

import paper_1003_1898_gb300 as P
from paper_1003_1898_gb300 import build, tune
from paper_1003_1898_gb300 import workloads as W


@pytest.mark.parametrize("gen", W.GENS)
@pytest.mark.parametrize("n", [1, 3, 4, 5, 4095, 4096, 4097, 65537, 10**7, 123456789])
def test_request_split_covers_n_with_aligned_rows(gen, n):
    s, per = W.request_split(gen, n)
    c = W.DRAWS_PER_STREAM.get(gen, W.DEFAULT_DRAWS_PER_STREAM)
    assert per % 4 == 0 and per > 0
    assert s * per >= n > (s - 1) * per          # no empty stream
    assert per <= 4 * -(-c // 4) + 4 or s == 1   # about C_g draws per stream


def test_batched_requests_mix():
    reqs = W.batched_requests(n_requests=20000)
    assert len(reqs) == 20000
    n = np.array([q["n"] for q in reqs])
    assert n.min() >= 100 and n.max() < 10**7
    # log-uniform lengths: about a fifth of the requests per decade
    dec = np.bincount(np.floor(np.log10(n)).astype(int) - 2, minlength=5)
    assert np.all(np.abs(dec / len(reqs) - 0.2) < 0.02)
    gens = {q["gen"] for q in reqs}
    assert gens == set(W.GENS)
    assert all(q["luxury"] == (W.BATCH_RANLUX_P if q["gen"] == "ranlux" else 0) for q in reqs)
    seeds = [q["seed"] for q in reqs]
    assert len(set(seeds)) == len(seeds)
    assert all(b - a == 1 << 32 for a, b in zip(seeds, seeds[1:]))   # disjoint stream ranges
    for q in reqs[:200]:
        assert (q["n_streams"], q["n_per"]) == W.request_split(q["gen"], q["n"])
    # deterministic
    assert W.batched_requests(n_requests=50) == W.batched_requests(n_requests=50)


def test_serving_workload():
    clients = W.serving_clients(512)
    assert len(clients) == 512
    assert sum(1 for g, lux, _ in clients if g == "ranlux" and lux == 223) == 256
    assert len({s for *_, s in clients}) == 512
    reqs = W.serving_requests(4000, rate=1000.0)
    t = np.array([r["arrival"] for r in reqs])
    assert np.all(np.diff(t) >= 0)
    assert abs(t[-1] / len(reqs) - 1e-3) < 1e-4          # Poisson at 1000 per second
    kinds = [r["kind"] for r in reqs]
    assert abs(kinds.count("ising") / len(reqs) - 0.5) < 0.05
    for r in reqs:
        if r["kind"] == "ising":
            assert r["L"] in W.SERVE_ISING_L and (r["L"] ** 2 // 2) % W.SERVE_STREAMS == 0
        else:
            assert 10**3 <= r["n"] <= 10**6


def test_jump_offsets_include_the_check_points():
    n, c = W.JUMP["n"], W.JUMP["n_chunks"]
    off = W.jump_offsets(n, c)
    assert len(off) >= 4096 and np.all(np.diff(off.astype(np.int64)) > 0)
    s = set(int(x) for x in off)
    L = -(-n // c)
    assert {0, 9999, n - 1} <= s
    assert all(k * L in s for k in range(0, c, 16))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return P.lib()


@pytest.mark.parametrize("ranlux_p", [24, 223])
def test_tile_table_accepts_compiled_tiles_only(lib, ranlux_p):
    for gen in P.GEN_NAMES:
        lux = ranlux_p if gen == "ranlux" else 0
        saved = P.prng_get_tile(gen, lux)
        try:
            for t in tune.tiles_for(gen, lux):
                P.prng_set_tile(gen, lux, *t)
                assert tuple(P.prng_get_tile(gen, lux)) == tuple(t)
            with pytest.raises(P.PrngError) as e:
                P.prng_set_tile(gen, lux, 96, 7, 3)
            assert e.value.code == -7
        finally:
            P.prng_set_tile(gen, lux, *saved)


def test_ranlux_ring_tiles_at_every_level(lib):
    # The per-row ring form (56 columns) is compiled for every luxury level,
    # single-staged only.
    for p in (24, 48, 97, 223, 389, 120, 240, 408):
        saved = P.prng_get_tile("ranlux", p)
        try:
            for t in ((64, 56, 1), (128, 56, 1), (256, 56, 1)):
                P.prng_set_tile("ranlux", p, *t)
                assert tuple(P.prng_get_tile("ranlux", p)) == t
            with pytest.raises(P.PrngError) as e:
                P.prng_set_tile("ranlux", p, 128, 56, 2)
            assert e.value.code == -7
        finally:
            P.prng_set_tile("ranlux", p, *saved)
    for t in tune.tiles_for("ranlux", 24):
        assert t[1] != 96, "the 96-column tile is for p >= 97 only"


def test_wide_ranlux_tile_only_at_high_luxury(lib):
    # The 96-column RANLUX tile is compiled for p >= 97 only.
    saved = P.prng_get_tile("ranlux", 24)
    try:
        with pytest.raises(P.PrngError) as e:
            P.prng_set_tile("ranlux", 24, 64, 96, 1)
        assert e.value.code == -7
    finally:
        P.prng_set_tile("ranlux", 24, *saved)
    for p in (97, 223, 389, 120, 240, 408):
        saved = P.prng_get_tile("ranlux", p)
        try:
            P.prng_set_tile("ranlux", p, 64, 96, 1)
            assert tuple(P.prng_get_tile("ranlux", p)) == (64, 96, 1)
        finally:
            P.prng_set_tile("ranlux", p, *saved)


def test_tuned_tiles_apply(lib):
    cache = tune.load()
    assert cache is not None
    tune.apply(cache)
    for key, v in cache.items():
        if key.startswith("ranlux_p"):
            got = P.prng_get_tile("ranlux", int(key[len("ranlux_p"):]))
        else:
            got = P.prng_get_tile(key)
        assert tuple(got) == tuple(v["tile"]), key
