"""Batched fills: one launch over many handles gives, request by request,
exactly the oracle's draws and exactly what each handle gives alone."""
import numpy as np
import pytest

import oracle
from tests import inputs

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


def _alloc(n, f32):
    return torch.full((max(n, 1) + 4,), -7, dtype=torch.float32 if f32 else torch.int32,
                      device="cuda")


def _oracle_request(q):
    ref = oracle.fill(q["gen"], q["seed"], q["n_streams"], q["n_per"], luxury=q["luxury"])
    flat = ref.reshape(-1)[:q["n"]]
    return oracle.to_f32(q["gen"], flat).view(np.uint32) if q["f32"] else flat


def _bits(t, n):
    return t[:n].cpu().numpy().view(np.uint32)


def test_batch_matches_oracle_mixed_requests():
    reqs = inputs.batched_requests(n_requests=400, seed=0xB47C, min_len=1, max_len=40000)
    handles, outs, fr = [], [], []
    try:
        for q in reqs:
            h = P.prng_create(q["gen"], 0, q["n_streams"], q["luxury"])
            handles.append(h)
            o = _alloc(q["n"], q["f32"])
            outs.append(o)
            fr.append({"st": h, "d_out": o, "n_per_stream": q["n_per"], "n_valid": q["n"],
                       "f32": q["f32"], "reseed": True, "seed": q["seed"]})
        b = P.prng_batch_create(fr)
        info = P.prng_batch_info(b)
        assert info["requests"] == len(reqs)
        assert info["numbers"] == sum(q["n"] for q in reqs)
        P.prng_batch_launch(b)
        torch.cuda.synchronize()
        for q, o in zip(reqs, outs):
            host = o.cpu().numpy()
            got = host.view(np.uint32)
            np.testing.assert_array_equal(got[:q["n"]], _oracle_request(q), err_msg=str(q))
            assert np.all(host[q["n"]:] == -7), "write past n_valid"
        P.prng_batch_destroy(b)
    finally:
        for h in handles:
            P.prng_destroy(h)


@pytest.mark.parametrize("lux", [24, 97, 389, 240])
def test_batch_continues_handles_like_solo_fills(lux):
    # Two handles per generator: one filled through a batch launched three
    # times (re-seeded only by creation), its twin by plain fills.
    specs = [(g, lux if g == "ranlux" else 0, ns, nper)
             for g, ns, nper in [("ggl", 37, 130), ("xor128", 129, 77), ("ranecu", 5, 1000),
                                 ("ranmar", 70, 150), ("ranlux", 131, 61), ("mt19937", 9, 700)]]
    hb, hs, outs, fr = [], [], [], []
    try:
        for g, lx, ns, nper in specs:
            a = P.prng_create(g, 4242, ns, lx)
            s = P.prng_create(g, 4242, ns, lx)
            hb.append(a)
            hs.append(s)
            o = torch.empty(ns * nper, dtype=torch.int32, device="cuda")
            outs.append(o)
            fr.append({"st": a, "d_out": o, "n_per_stream": nper})
        b = P.prng_batch_create(fr)
        for launch in range(3):
            P.prng_batch_launch(b)
            torch.cuda.synchronize()
            for (g, lx, ns, nper), s, o in zip(specs, hs, outs):
                want = torch.empty(ns * nper, dtype=torch.int32, device="cuda")
                P.prng_fill_u32(s, want, nper)
                torch.cuda.synchronize()
                assert torch.equal(o, want), (g, launch)
        P.prng_batch_destroy(b)
    finally:
        for h in hb + hs:
            P.prng_destroy(h)


def test_batch_reseed_is_deterministic_across_launches():
    reqs = inputs.batched_requests(n_requests=60, seed=77, min_len=50, max_len=5000)
    handles, outs, fr = [], [], []
    try:
        for q in reqs:
            h = P.prng_create(q["gen"], 1, q["n_streams"], q["luxury"])
            handles.append(h)
            o = _alloc(q["n"], q["f32"])
            outs.append(o)
            fr.append({"st": h, "d_out": o, "n_per_stream": q["n_per"], "n_valid": q["n"],
                       "f32": q["f32"], "reseed": True, "seed": q["seed"]})
        b = P.prng_batch_create(fr)
        P.prng_batch_launch(b)
        torch.cuda.synchronize()
        first = [o.clone() for o in outs]
        for _ in range(3):
            P.prng_batch_launch(b)
        torch.cuda.synchronize()
        for a, o in zip(first, outs):
            assert torch.equal(a, o)
        P.prng_batch_destroy(b)
    finally:
        for h in handles:
            P.prng_destroy(h)


def test_batch_rejects_duplicate_handle():
    h = P.prng_create("ggl", 1, 4, 0)
    o = torch.empty(64, dtype=torch.int32, device="cuda")
    try:
        with pytest.raises(P.PrngError) as e:
            P.prng_batch_create([{"st": h, "d_out": o, "n_per_stream": 8},
                                 {"st": h, "d_out": o, "n_per_stream": 8}])
        assert e.value.code == -8
    finally:
        P.prng_destroy(h)


def test_batcher_launches_continue_streams_and_reject_duplicates():
    # The serving loop's batcher: repeated launches over resident handles
    # continue every stream; a handle twice in one launch, or more requests
    # than the batcher was sized for, is rejected before anything runs.
    specs = [("ggl", 0), ("ranlux", 223), ("mt19937", 0), ("ranmar", 0)]
    ns, per = 64, 40
    handles = [P.prng_create(g, 900 + i, ns, lux) for i, (g, lux) in enumerate(specs)]
    b = P.prng_batcher_create(4, 4096)
    try:
        outs = [[_alloc(ns * per, False) for _ in specs] for _ in range(2)]
        for t in range(2):
            P.prng_batcher_launch(b, [{"st": h, "d_out": o, "n_per_stream": per}
                                      for h, o in zip(handles, outs[t])])
        torch.cuda.synchronize()
        for i, (g, lux) in enumerate(specs):
            ref = oracle.fill(g, 900 + i, ns, 2 * per, luxury=lux)
            for t in range(2):
                got = _bits(outs[t][i], ns * per).reshape(ns, per)
                np.testing.assert_array_equal(got, ref[:, t * per:(t + 1) * per], err_msg=g)
        o = _alloc(ns * per, False)
        with pytest.raises(P.PrngError) as e:
            P.prng_batcher_launch(b, [{"st": handles[0], "d_out": o, "n_per_stream": per},
                                      {"st": handles[0], "d_out": o, "n_per_stream": per}])
        assert e.value.code == -8
        with pytest.raises(P.PrngError) as e:
            P.prng_batcher_launch(b, [{"st": h, "d_out": o, "n_per_stream": per}
                                      for h in handles + [handles[0]]])
        assert e.value.code == -3
    finally:
        P.prng_batcher_destroy(b)
        for h in handles:
            P.prng_destroy(h)
