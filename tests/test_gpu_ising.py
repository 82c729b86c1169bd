"""Checkerboard Ising runs driven by the library's draws: lattice, energy and
magnetisation after every sweep equal the oracle's."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1003_1898_gb300 as P  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_1898_gb300 import build
    build.build()
    P.lib()


def gpu_ising_run(gen, seed, n_streams, L, sweeps, lux=0, beta=oracle.ISING_BETA):
    t4, t8 = P.prng_ising_thresholds(beta)
    assert (t4, t8) == oracle.ising_thresholds(beta)
    h = P.prng_create(gen, seed, n_streams, lux)
    spins = torch.ones((L, L), dtype=torch.int8, device="cuda")
    draws = torch.empty(L * L // 2, dtype=torch.int32, device="cuda")
    per = L * L // (2 * n_streams)
    em = []
    try:
        for sw in range(sweeps):
            for colour in (0, 1):
                P.prng_fill_u32(h, draws, per)
                P.prng_ising_half_sweep([{"d_spins": spins, "d_draws": draws, "L": L,
                                          "colour": colour, "gen": gen, "t4": t4, "t8": t8}])
            s = spins.cpu().numpy()
            em.append((oracle.ising_energy(s), oracle.ising_magnetisation(s)))
    finally:
        P.prng_destroy(h)
    return spins.cpu().numpy(), em


@pytest.mark.parametrize("gen,lux", [("ggl", 0), ("xor128", 0), ("ranecu", 0), ("ranmar", 0),
                                     ("ranlux", 223), ("mt19937", 0)])
@pytest.mark.parametrize("L,ns", [(64, 32), (96, 48)])
def test_ising_run_equals_oracle(gen, lux, L, ns):
    got, em = gpu_ising_run(gen, 321, ns, L, 6, lux)
    want, em_want = oracle.ising_run(gen, 321, ns, L, 6, luxury=lux)
    np.testing.assert_array_equal(got, want)
    assert em == em_want


def test_several_lattices_in_one_launch():
    t4, t8 = P.prng_ising_thresholds(0.3)
    rng = np.random.default_rng(3)
    sizes = [8, 30, 64, 128, 256, 2]
    lat, draws, want = [], [], []
    for L in sizes:
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, L))
        d = rng.integers(0, 2**32, size=L * L // 2, dtype=np.uint64).astype(np.uint32)
        lat.append(torch.from_numpy(s.copy()).cuda())
        draws.append(torch.from_numpy(d.view(np.int32)).cuda())
        w = s.copy()
        oracle.ising_half_sweep(w, d, "mt19937", 1, t4, t8)
        want.append(w)
    P.prng_ising_half_sweep([{"d_spins": a, "d_draws": b, "L": L, "colour": 1, "gen": "mt19937",
                              "t4": t4, "t8": t8} for a, b, L in zip(lat, draws, sizes)])
    torch.cuda.synchronize()
    for a, w in zip(lat, want):
        np.testing.assert_array_equal(a.cpu().numpy(), w)


@pytest.mark.parametrize("colour", [0, 1])
def test_vector_and_scalar_forms_in_one_call(colour):
    # L multiple of 16 takes the 16-site vector form, the others the scalar
    # form; pitched draw rows (per % 8 == 0) stay on the vector form.
    t4, t8 = P.prng_ising_thresholds(0.25)
    rng = np.random.default_rng(11 + colour)
    cases = [(16, 0, 0), (48, 0, 0), (256, 0, 0), (1024, 64, 3 * 64), (96, 72, 2 * 72),
             (34, 0, 0), (64, 2, 6), (130, 0, 0)]
    lat, bufs, reqs, want = [], [], [], []
    for L, per, pitch in cases:
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, L))
        n = L * L // 2
        if pitch:
            rows = n // per
            buf = rng.integers(0, 2**32, size=rows * pitch, dtype=np.uint64).astype(np.uint32)
            k = np.arange(n)
            d = buf[(k // per) * pitch + k % per]
        else:
            buf = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
            d = buf
        a = torch.from_numpy(s.copy()).cuda()
        b = torch.from_numpy(buf.view(np.int32).copy()).cuda()
        lat.append(a)
        bufs.append(b)
        reqs.append({"d_spins": a, "d_draws": b, "L": L, "colour": colour, "gen": "xor128",
                     "t4": t4, "t8": t8, "per": per, "pitch": pitch})
        w = s.copy()
        oracle.ising_half_sweep(w, d, "xor128", colour, t4, t8)
        want.append(w)
    P.prng_ising_half_sweep(reqs)
    torch.cuda.synchronize()
    for a, w, c in zip(lat, want, cases):
        np.testing.assert_array_equal(a.cpu().numpy(), w, err_msg=str(c))


def test_ising_rejects_bad_lattices():
    d = torch.empty(8, dtype=torch.int32, device="cuda")
    s = torch.ones((4, 4), dtype=torch.int8, device="cuda")
    with pytest.raises(P.PrngError):
        P.prng_ising_half_sweep([{"d_spins": s, "d_draws": d, "L": 3, "colour": 0, "shift": 0,
                                  "t4": 0, "t8": 0}])
    with pytest.raises(P.PrngError):
        P.prng_ising_half_sweep([{"d_spins": s, "d_draws": d, "L": 4, "colour": 2, "shift": 0,
                                  "t4": 0, "t8": 0}])


# ------------------------------------------------------------ fused half-sweeps

def gpu_fused_run(gen, seed, n_streams, L, sweeps, lux=0, beta=oracle.ISING_BETA):
    t4, t8 = P.prng_ising_thresholds(beta)
    h = P.prng_create(gen, seed, n_streams, lux)
    spins = torch.ones((L, L), dtype=torch.int8, device="cuda")
    em = []
    try:
        for sw in range(sweeps):
            for colour in (0, 1):
                P.prng_ising_fused(h, spins, L, colour, t4, t8)
            s = spins.cpu().numpy()
            em.append((oracle.ising_energy(s), oracle.ising_magnetisation(s)))
    finally:
        P.prng_destroy(h)
    return spins.cpu().numpy(), em


@pytest.mark.parametrize("gen,lux", [("ggl", 0), ("xor128", 0), ("ranecu", 0), ("ranmar", 0),
                                     ("ranlux", 223), ("ranlux", 24), ("mt19937", 0)])
@pytest.mark.parametrize("L,ns", [(64, 32), (96, 48), (256, 1024), (130, 65)])
def test_fused_run_equals_oracle(gen, lux, L, ns):
    # Draws consumed where they are made give the same lattice after every
    # sweep as the stored draws and the oracle.
    got, em = gpu_fused_run(gen, 321, ns, L, 5, lux)
    want, em_want = oracle.ising_run(gen, 321, ns, L, 5, luxury=lux)
    np.testing.assert_array_equal(got, want)
    assert em == em_want


@pytest.mark.parametrize("gen", ["ggl", "xor128", "ranmar", "mt19937"])
def test_fused_then_fill_continues_the_stream(gen):
    # A fused half-sweep advances the handle like the fill it replaces.
    L, ns = 64, 32
    t4, t8 = P.prng_ising_thresholds(0.44)
    a = P.prng_create(gen, 9, ns, 0)
    b = P.prng_create(gen, 9, ns, 0)
    try:
        P.prng_ising_fused(a, torch.ones((L, L), dtype=torch.int8, device="cuda"), L, 0, t4, t8)
        P.prng_skip(b, L * L // (2 * ns))
        x = torch.empty(ns * 50, dtype=torch.int32, device="cuda")
        y = torch.empty(ns * 50, dtype=torch.int32, device="cuda")
        P.prng_fill_u32(a, x, 50)
        P.prng_fill_u32(b, y, 50)
        torch.cuda.synchronize()
        assert torch.equal(x, y)
    finally:
        P.prng_destroy(a)
        P.prng_destroy(b)


def test_fused_rejects_bad_shapes():
    h = P.prng_create("ggl", 1, 48, 0)
    s = torch.ones((64, 64), dtype=torch.int8, device="cuda")
    try:
        for L, colour in [(63, 0), (64, 2), (0, 0), (10, 0)]:     # odd, colour, empty, 50 % 48
            with pytest.raises(P.PrngError):
                P.prng_ising_fused(h, s, L, colour, 1, 1)
    finally:
        P.prng_destroy(h)
