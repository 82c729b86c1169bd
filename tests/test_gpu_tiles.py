"""Every launch tile compiled into the library gives the oracle's output
(the autotuner may pick any of them)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1003_1898_gb300 as P  # noqa: E402
from paper_1003_1898_gb300 import tune  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_1898_gb300 import build
    build.build()
    P.lib()


CASES = [(g, t, 223 if g == "ranlux" else 0) for g in P.GEN_NAMES
         for t in tune.tiles_for(g, 223 if g == "ranlux" else 0)]
CASES += [("ranlux", t, 24) for t in tune.tiles_for("ranlux", 24)]


@pytest.mark.parametrize("gen,tile,lux", CASES,
                         ids=[f"{g}-{'x'.join(map(str, t))}-p{p}" for g, t, p in CASES])
def test_tile_parity(gen, tile, lux):
    saved = P.prng_get_tile(gen, lux)
    P.prng_set_tile(gen, lux, *tile)
    try:
        ns = 301                                   # > 2 CTAs of 128, ragged last CTA, odd
        pieces = [700, 64, 33, 1300]               # continuation across fills, ragged tails
        total = sum(pieces)
        ref = oracle.fill(gen, 77, ns, total, luxury=lux)
        h = P.prng_create(gen, 77, ns, lux)
        try:
            col = 0
            for i, k in enumerate(pieces):
                f32 = i % 2 == 1
                out = torch.empty(ns * k, dtype=torch.float32 if f32 else torch.int32, device="cuda")
                (P.prng_fill_f32 if f32 else P.prng_fill_u32)(h, out, k)
                torch.cuda.synchronize()
                got = out.cpu().numpy().reshape(ns, k).view(np.uint32)
                want = ref[:, col:col + k]
                if f32:
                    want = oracle.to_f32(gen, want).view(np.uint32)
                np.testing.assert_array_equal(got, want, err_msg=f"piece {i}")
                col += k
        finally:
            P.prng_destroy(h)
    finally:
        P.prng_set_tile(gen, lux, *saved)


@pytest.mark.parametrize("lux,tile", [(24, (128, 56, 1)), (24, (64, 56, 1)), (24, (256, 56, 1)),
                                      (48, (128, 56, 1)), (223, (128, 56, 1)), (223, (64, 56, 1))])
def test_ranlux_ring_positions(lux, tile):
    # Fills whose start positions and lengths reach every branch of the ring
    # form: fills that end inside the open block (4 draws, and 2), heads of
    # 4..20 draws, copy-outs from every ring offset, tails of 1..23 draws;
    # interleaved with fills that the launcher hands to the tiled form (odd
    # lengths: a row pitch, or a start position, that is not a multiple of 4).
    pieces = [8, 4, 2, 10, 100, 4, 76, 1, 3, 48, 252, 24, 5, 96, 1000, 12, 7, 1024, 20, 32, 56, 60]
    ns = 301
    saved = P.prng_get_tile("ranlux", lux)
    P.prng_set_tile("ranlux", lux, *tile)
    try:
        ref = oracle.fill("ranlux", 91, ns, sum(pieces), luxury=lux)
        h = P.prng_create("ranlux", 91, ns, lux)
        try:
            col = 0
            for i, k in enumerate(pieces):
                f32 = i % 3 == 2
                out = torch.full((ns * k + 4,), -7, dtype=torch.int32, device="cuda")
                (P.prng_fill_f32 if f32 else P.prng_fill_u32)(h, out, k)
                torch.cuda.synchronize()
                got = out[:ns * k].cpu().numpy().reshape(ns, k).view(np.uint32)
                want = ref[:, col:col + k]
                if f32:
                    want = oracle.to_f32("ranlux", want).view(np.uint32)
                np.testing.assert_array_equal(got, want, err_msg=f"piece {i} ({k} draws)")
                assert np.all(out[ns * k:].cpu().numpy() == -7), f"piece {i} wrote past its rows"
                col += k
        finally:
            P.prng_destroy(h)
    finally:
        P.prng_set_tile("ranlux", lux, *saved)


@pytest.mark.parametrize("gen", ["ggl", "ranecu"])
@pytest.mark.parametrize("tile", tune.TILES["ggl"])
def test_tile_parity_jump(gen, tile):
    # Lane-parallel tiles run a warp per chunk; staged tiles a thread per
    # (possibly finer) chunk started by a^(row L) x0.
    saved = P.prng_get_tile(gen)
    P.prng_set_tile(gen, 0, *tile)
    try:
        x0 = 1 if gen == "ggl" else (1 | (1 << 32))
        n = 123457
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        P.prng_fill_jump_u32(gen, x0, n, 333, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), oracle.serial_fill(gen, x0, n))
    finally:
        P.prng_set_tile(gen, 0, *saved)


@pytest.mark.parametrize("tile", tune.TILES["mt19937"])
def test_tile_parity_mt_jump(tile):
    # 37 chunk rows (odd: with two streams per warp the last warp has an
    # idle half) and a last row cut short by the element limit.
    saved = P.prng_get_tile("mt19937")
    P.prng_set_tile("mt19937", 0, *tile)
    try:
        n = 100003
        out = torch.full((n + 4,), -7, dtype=torch.int32, device="cuda")
        P.prng_fill_jump_u32("mt19937", 5489, n, 37, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got[:n], oracle.serial_fill("mt19937", 5489, n))
        assert np.all(got[n:] == np.uint32(2**32 - 7)), "write past the end"
    finally:
        P.prng_set_tile("mt19937", 0, *saved)


@pytest.mark.parametrize("tile", tune.TILES["mt19937"])
def test_tile_parity_mt_f64_and_fused(tile):
    # The MT19937 tiles on the other output modes: doubles from pairs (whole
    # 624-word blocks, so the register-resident block loop of the half-warp
    # tiles runs) and the fused Ising half-sweep (whole and partial blocks).
    saved = P.prng_get_tile("mt19937")
    P.prng_set_tile("mt19937", 0, *tile)
    try:
        ns, nd = 37, 1300                          # 2600 draws: four whole blocks and a tail
        h = P.prng_create("mt19937", 91, ns, 0)
        try:
            out = torch.empty(ns * nd, dtype=torch.float64, device="cuda")
            P.prng_fill_f64(h, out, nd)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy().reshape(ns, nd),
                                          oracle.fill_f64("mt19937", 91, ns, nd))
        finally:
            P.prng_destroy(h)
        t4, t8 = P.prng_ising_thresholds(oracle.ISING_BETA)
        L, ns = 256, 32                            # 1024 draws per stream per half-sweep
        h = P.prng_create("mt19937", 92, ns, 0)
        try:
            spins = torch.ones((L, L), dtype=torch.int8, device="cuda")
            for _ in range(3):
                for colour in (0, 1):
                    P.prng_ising_fused(h, spins, L, colour, t4, t8)
            torch.cuda.synchronize()
            want, _ = oracle.ising_run("mt19937", 92, ns, L, 3)
            np.testing.assert_array_equal(spins.cpu().numpy(), want)
        finally:
            P.prng_destroy(h)
    finally:
        P.prng_set_tile("mt19937", 0, *saved)
