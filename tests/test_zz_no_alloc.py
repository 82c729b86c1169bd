"""The allocation-free batched fill (prng_batch_fill_noalloc) against the
allocating one (prng_batch_create / prng_batch_launch).

prng_batch_fill_noalloc exists for callers that must not let the library
allocate device memory (a framework's caching allocator, memory reserved up
front, loops that cannot afford an allocation's synchronisation); its
scratch is a fixed device array inside the library.  Twin handles are
filled by both entry points, twice in a row, and every output must be the
same bytes.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1003_1898_gb300 as P  # noqa: E402

SPECS = [("ggl", 0, 33, 130), ("xor128", 0, 129, 77), ("ranecu", 0, 7, 1000),
         ("ranmar", 0, 70, 150), ("ranlux", 223, 131, 61), ("ranlux", 24, 5, 100),
         ("ranlux", 408, 3, 50), ("mt19937", 0, 9, 700)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_1898_gb300 import build
    build.build()
    P.lib()


def _setup():
    a_handles, b_handles, a_out, b_out, a_req, b_req = [], [], [], [], [], []
    for i, (g, lux, ns, nper) in enumerate(SPECS):
        a = P.prng_create(g, 900 + i, ns, lux)
        b = P.prng_create(g, 900 + i, ns, lux)
        P.prng_skip(a, 13)          # leave RANLUX / MT19937 inside a block
        P.prng_skip(b, 13)
        f32 = i % 2 == 1
        oa = torch.full((ns * nper + 4,), -7, dtype=torch.float32 if f32 else torch.int32, device="cuda")
        ob = oa.clone()
        n_valid = ns * nper - (nper // 3)            # last stream only partly wanted
        for h, o, hs, outs, reqs in ((a, oa, a_handles, a_out, a_req), (b, ob, b_handles, b_out, b_req)):
            hs.append(h)
            outs.append(o)
            reqs.append({"st": h, "d_out": o, "n_per_stream": nper, "n_valid": n_valid, "f32": f32})
    return a_handles, b_handles, a_out, b_out, a_req, b_req


def test_noalloc_batch_equals_allocating_batch_two_calls():
    a_h, b_h, a_out, b_out, a_req, b_req = _setup()
    try:
        for call in range(2):
            reseed = call == 1                       # second call also re-seeds from a new base
            for ra, rb in zip(a_req, b_req):
                ra["reseed"] = rb["reseed"] = reseed
                ra["seed"] = rb["seed"] = 5000 + call
            P.prng_batch_fill_noalloc(a_req)
            b = P.prng_batch_create(b_req)
            P.prng_batch_launch(b)
            torch.cuda.synchronize()
            P.prng_batch_destroy(b)
            for (g, lux, ns, nper), oa, ob in zip(SPECS, a_out, b_out):
                assert np.array_equal(oa.cpu().numpy().view(np.uint32), ob.cpu().numpy().view(np.uint32)), \
                    (g, lux, call)
            # and both are the oracle's draws: call 0 continues each stream
            # after its 13 skipped draws, call 1 re-seeds from 5001
            for i, ((g, lux, ns, nper), oa, ra) in enumerate(zip(SPECS, a_out, a_req)):
                seed, skip = (900 + i, 13) if call == 0 else (5001, 0)
                ref = oracle.fill(g, seed, ns, nper, luxury=lux, skip=skip).reshape(-1)
                if ra["f32"]:
                    ref = oracle.to_f32(g, ref).view(np.uint32)
                n = ra["n_valid"]
                host = oa.cpu().numpy()
                assert np.array_equal(host.view(np.uint32)[:n], ref[:n]), (g, lux, call)
                assert np.all(host[n:] == -7), (g, lux, call, "wrote past n_valid")
        # the handles themselves advanced identically
        for ha, hb in zip(a_h, b_h):
            assert P.prng_get_state(ha) == P.prng_get_state(hb)
    finally:
        for h in a_h + b_h:
            P.prng_destroy(h)


def test_noalloc_rejects_batches_beyond_its_scratch():
    L = P.lib()
    h = P.prng_create("ggl", 1, 1, 0)
    try:
        n = 4097                                     # PRNG_NOALLOC_MAX_REQUESTS + 1
        arr = (P.PrngFillReq * n)()
        assert L.prng_batch_fill_noalloc(arr, n, None) == -10
        assert "scratch" in P.prng_strerror(-10)
        # too many work items: one request whose streams exceed the item limit
        big = P.prng_create("xor128", 1, 131073 * 128, 0)
        try:
            one = (P.PrngFillReq * 1)()
            one[0].st = big.value
            one[0].d_out = 16
            one[0].n_per_stream = 1
            assert L.prng_batch_fill_noalloc(one, 1, None) == -10
        finally:
            P.prng_destroy(big)
    finally:
        P.prng_destroy(h)
