"""Oracle parity at the full sizes of the batched and serving workloads.

* Batched: the whole 20,000-request workload (lengths log-uniform in
  [10^2, 10^7], the six generators, RANLUX at p = 223, u32 or f32; about
  1.75e10 numbers in 486,000 work items) runs as one batch launch, and a
  seeded sample of requests -- always including the longest request of each
  generator -- is compared with the oracle on its first, middle and last
  streams, including the element cut at n_valid.
* Serving: checkerboard Ising runs at the serving sizes (L = 1024 for 16
  sweeps, L = 4096 for 2 sweeps) on a serving client's streams, with the draws
  stored (fill, then half-sweep) and consumed where they are made (fused),
  against the oracle's lattice, energy and magnetisation after every sweep.
"""
import functools

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1003_1898_gb300 as P  # noqa: E402
from paper_1003_1898_gb300 import workloads as W  # noqa: E402

SENTINEL = -7


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_1898_gb300 import build
    build.build()
    P.lib()


def _sampled_requests(reqs, k=240, seed=0xC0F4):
    """k request indices drawn with a fixed seed, plus the longest request
    of each generator."""
    rng = np.random.default_rng(seed)
    pick = set(int(i) for i in rng.choice(len(reqs), size=k, replace=False))
    for g in W.GENS:
        idx = [i for i, q in enumerate(reqs) if q["gen"] == g]
        pick.add(max(idx, key=lambda i: reqs[i]["n"]))
    return sorted(pick)


def test_batched_workload_full_size_matches_oracle():
    reqs = W.batched_requests()
    assert len(reqs) == 20000
    sizes = [((q["n_streams"] * q["n_per"] + 3) // 4) * 4 for q in reqs]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    buf = torch.full((int(offs[-1]),), SENTINEL, dtype=torch.int32, device="cuda")
    base = buf.data_ptr()
    handles = []
    b = None
    try:
        for q in reqs:
            handles.append(P.prng_create(q["gen"], 0, q["n_streams"], q["luxury"]))
        fr = [{"st": h, "d_out": base + 4 * int(o), "n_per_stream": q["n_per"], "n_valid": q["n"],
               "f32": q["f32"], "reseed": True, "seed": q["seed"]}
              for h, q, o in zip(handles, reqs, offs[:-1])]
        b = P.prng_batch_create(fr)
        info = P.prng_batch_info(b)
        assert info["numbers"] == sum(q["n"] for q in reqs)
        assert info["items"] > 400000
        P.prng_batch_launch(b)
        torch.cuda.synchronize()
        checked = 0
        for i in _sampled_requests(reqs):
            q = reqs[i]
            ns, per, n = q["n_streams"], q["n_per"], q["n"]
            rows = sorted({0, ns // 2, ns - 1})
            for r in rows:
                lo = int(offs[i]) + r * per
                width = min(per, n - r * per)          # the last row may be cut at n_valid
                got = buf[lo: lo + per].cpu().numpy().view(np.uint32)
                ref = oracle.fill(q["gen"], q["seed"], 1, per, luxury=q["luxury"], stream0=r)[0]
                if q["f32"]:
                    ref = oracle.to_f32(q["gen"], ref).view(np.uint32)
                np.testing.assert_array_equal(got[:width], ref[:width],
                                              err_msg=f"request {i} {q['gen']} row {r}")
                assert np.all(got[width:].view(np.int32) == SENTINEL), f"request {i} wrote past n"
            tail = buf[int(offs[i]) + n: int(offs[i + 1])].cpu().numpy()
            assert np.all(tail == SENTINEL), f"request {i} wrote past n_valid"
            checked += 1
        assert checked >= 200
    finally:
        if b is not None:
            P.prng_batch_destroy(b)
        for h in handles:
            P.prng_destroy(h)
        del buf
        torch.cuda.empty_cache()


# ------------------------------------------------------------ Ising at serving sizes

STREAMS = W.SERVE_STREAMS


@functools.lru_cache(maxsize=None)
def _oracle_run(gen, lux, L, sweeps):
    return oracle.ising_run(gen, 0xA5 + L, STREAMS, L, sweeps, luxury=lux)


def _gpu_run(gen, lux, L, sweeps, fused):
    t4, t8 = P.prng_ising_thresholds(oracle.ISING_BETA)
    h = P.prng_create(gen, 0xA5 + L, STREAMS, lux)
    spins = torch.ones((L, L), dtype=torch.int8, device="cuda")
    draws = None if fused else torch.empty(L * L // 2, dtype=torch.int32, device="cuda")
    per = L * L // (2 * STREAMS)
    em = []
    try:
        for _ in range(sweeps):
            for colour in (0, 1):
                if fused:
                    P.prng_ising_fused(h, spins, L, colour, t4, t8)
                else:
                    P.prng_fill_u32(h, draws, per)
                    P.prng_ising_half_sweep([{"d_spins": spins, "d_draws": draws, "L": L,
                                              "colour": colour, "gen": gen, "t4": t4, "t8": t8}])
            s = spins.cpu().numpy()
            em.append((oracle.ising_energy(s), oracle.ising_magnetisation(s)))
    finally:
        P.prng_destroy(h)
    return spins.cpu().numpy(), em


CASES = [(g, 223 if g == "ranlux" else 0, 1024, W.SERVE_SWEEPS) for g in W.GENS] + \
        [(g, lux, 4096, 2) for g, lux in (("ggl", 0), ("ranlux", 223), ("mt19937", 0))]


@pytest.mark.parametrize("fused", [False, True], ids=["stored", "fused"])
@pytest.mark.parametrize("gen,lux,L,sweeps", CASES, ids=lambda v: str(v))
def test_ising_serving_sizes_equal_oracle(gen, lux, L, sweeps, fused):
    got, em = _gpu_run(gen, lux, L, sweeps, fused)
    want, em_want = _oracle_run(gen, lux, L, sweeps)
    np.testing.assert_array_equal(got, want)
    assert em == em_want
