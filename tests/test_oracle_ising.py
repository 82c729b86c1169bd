"""Pins of the oracle's checkerboard Ising consumer (no GPU)."""
import math

import numpy as np
import pytest

import oracle


def test_thresholds_are_floor_of_boltzmann_weights():
    t4, t8 = oracle.ising_thresholds(0.4406868)
    assert t4 == math.floor(2**24 * math.exp(-4 * 0.4406868))
    assert t8 == math.floor(2**24 * math.exp(-8 * 0.4406868))
    assert oracle.ising_thresholds(0.0) == (2**24, 2**24)


def test_closed_forms_of_the_ordered_lattice():
    for L in (4, 16, 64):
        s = np.ones((L, L), dtype=np.int8)
        assert oracle.ising_energy(s) == -2 * L * L
        assert oracle.ising_magnetisation(s) == L * L
        s[::2, ::2] *= -1
        s[1::2, 1::2] *= -1                     # checkerboard: every bond unsatisfied
        assert oracle.ising_energy(s) == 2 * L * L
        assert oracle.ising_magnetisation(s) == 0


def test_infinite_temperature_flips_every_site():
    # beta = 0: both thresholds are 2^24, every proposal is accepted, so each
    # half-sweep flips its whole colour; from all +1 the lattice alternates.
    L = 16
    s, em = oracle.ising_run("xor128", 3, 8, L, 6, beta=0.0)
    for k, (e, m) in enumerate(em):
        assert e == -2 * L * L
        assert m == (-1) ** (k + 1) * L * L


def test_zero_temperature_never_raises_the_energy():
    L = 32
    rng = np.random.default_rng(5)
    s = rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, L))
    t4, t8 = 0, 0                            # beta -> infinity: only dE <= 0 accepted
    draws = rng.integers(0, 2**32, size=L * L // 2, dtype=np.uint64).astype(np.uint32)
    e_prev = oracle.ising_energy(s)
    for h in range(40):
        oracle.ising_half_sweep(s, draws, "mt19937", h % 2, t4, t8)
        e = oracle.ising_energy(s)
        assert e <= e_prev
        e_prev = e
    cold = np.ones((L, L), dtype=np.int8)
    oracle.ising_half_sweep(cold, draws, "mt19937", 0, 0, 0)
    assert np.all(cold == 1)


def _numpy_half_sweep(s, draws, sh, colour, t4, t8):
    # Same rule through whole-array operations: neighbour sums by periodic
    # rolls, the colour mask, and the draws placed on their sites.
    L = s.shape[0]
    nb = (np.roll(s, 1, 0) + np.roll(s, -1, 0) + np.roll(s, 1, 1) + np.roll(s, -1, 1)).astype(np.int32)
    dE = 2 * s.astype(np.int32) * nb
    y, x = np.indices((L, L))
    mask = (x + y) % 2 == colour
    r = np.zeros((L, L), dtype=np.uint64)
    r[mask] = (draws.astype(np.uint64) >> np.uint64(sh))  # row-major order of the colour's sites
    acc = (dE <= 0) | ((dE == 4) & (r < t4)) | ((dE == 8) & (r < t8))
    out = s.copy()
    out[mask & acc] = -s[mask & acc]
    return out


@pytest.mark.parametrize("gen", ["ggl", "ranmar", "mt19937"])
def test_half_sweep_equals_array_formulation(gen):
    rng = np.random.default_rng(11)
    L = 12
    s = rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, L))
    t4, t8 = oracle.ising_thresholds(0.35)
    sh = oracle.SHIFT[oracle.gen_id(gen)]
    for h in range(10):
        draws = rng.integers(0, 2**32, size=L * L // 2, dtype=np.uint64).astype(np.uint32)
        want = _numpy_half_sweep(s, draws, sh, h % 2, t4, t8)
        oracle.ising_half_sweep(s, draws, gen, h % 2, t4, t8)
        np.testing.assert_array_equal(s, want)


def _onsager_energy(beta):
    from scipy.special import ellipk
    k = 2 * math.sinh(2 * beta) / math.cosh(2 * beta) ** 2
    th = math.tanh(2 * beta)
    return -(1 / math.tanh(2 * beta)) * (1 + (2 / math.pi) * (2 * th * th - 1) * ellipk(k * k))


@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_energy_matches_onsager_away_from_criticality(beta):
    # Physics sanity: the equilibrium energy per site of the infinite lattice
    # (Onsager) at temperatures where L = 64 is many correlation lengths.
    pytest.importorskip("scipy")
    L, burn, meas = 64, 300, 700
    s, em = oracle.ising_run("xor128", 2024, 64, L, burn + meas, beta=beta)
    e = np.mean([x[0] for x in em[burn:]]) / (L * L)
    assert abs(e - _onsager_energy(beta)) < 0.01
