"""Fills whose output is host memory from prng_host_alloc: the kernels store
straight into mapped page-locked memory.  Same bar as device outputs:
bit-exact against the oracle, nothing written outside the output."""
import numpy as np
import pytest

import oracle
from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1003_1898_gb300 as P  # noqa: E402

SENT = np.uint32(0xA5A5A5A5)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_1898_gb300 import build
    build.build()
    P.lib()


def host_buf(n_words, pad=16):
    """Host buffer of n_words + 2 pad words of sentinel; the output starts
    pad words in (16-byte aligned)."""
    b = P.HostBuffer(4 * (n_words + 2 * pad))
    b.numpy("uint32")[:] = SENT
    return b, b.ptr + 4 * pad


def check_pads(b, n_words, pad=16):
    w = b.numpy("uint32")
    assert np.all(w[:pad] == SENT), "write before the start"
    assert np.all(w[pad + n_words:] == SENT), "write past the end"
    return w[pad:pad + n_words]


def test_host_alloc_pointer_is_device_addressable():
    b = P.HostBuffer(1 << 20)
    try:
        t = torch.arange(1 << 18, dtype=torch.int32, device="cuda")
        h = P.prng_create("ggl", 1, 256)
        P.prng_fill_u32(h, b.ptr, 1024)
        torch.cuda.synchronize()
        P.prng_destroy(h)
        assert b.numpy("uint32").size == 1 << 18
        del t
    finally:
        b.close()


@pytest.mark.parametrize("gen", inputs.GENS)
@pytest.mark.parametrize("dtype", ["u32", "f32", "f64"])
def test_fill_into_host_every_element(gen, dtype):
    ns, nper = 257, 1000
    lux = 223 if gen == "ranlux" else 0
    words = ns * nper * (2 if dtype == "f64" else 1)
    b, out = host_buf(words)
    h = P.prng_create(gen, 31, ns, lux)
    try:
        {"u32": P.prng_fill_u32, "f32": P.prng_fill_f32, "f64": P.prng_fill_f64}[dtype](h, out, nper)
        torch.cuda.synchronize()
        got = check_pads(b, words)
        if dtype == "f64":
            ref = oracle.fill_f64(gen, 31, ns, nper, luxury=lux).reshape(-1).view(np.uint32)
        else:
            ru = oracle.fill(gen, 31, ns, nper, luxury=lux).reshape(-1)
            ref = oracle.to_f32(gen, ru).view(np.uint32) if dtype == "f32" else ru
        np.testing.assert_array_equal(got, ref)
    finally:
        P.prng_destroy(h)
        b.close()


@pytest.mark.parametrize("gen", ["ggl", "ranecu", "xor128", "mt19937"])
def test_jump_fill_into_host(gen):
    n, chunks = 100003, 37
    x0 = inputs.JUMP_X0[gen]
    b, out = host_buf(n)
    try:
        P.prng_fill_jump_u32(gen, x0, n, chunks, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(check_pads(b, n), oracle.serial_fill(gen, x0, n))
    finally:
        b.close()


def test_batched_requests_into_host():
    reqs = inputs.batched_requests(n_requests=60, seed=0x4057, min_len=1, max_len=20000)
    handles, bufs, fr = [], [], []
    try:
        for q in reqs:
            h = P.prng_create(q["gen"], 0, q["n_streams"], q["luxury"])
            handles.append(h)
            b, out = host_buf(q["n"])
            bufs.append(b)
            fr.append({"st": h, "d_out": out, "n_per_stream": q["n_per"], "n_valid": q["n"],
                       "f32": q["f32"], "reseed": True, "seed": q["seed"]})
        bt = P.prng_batch_create(fr)
        P.prng_batch_launch(bt)
        torch.cuda.synchronize()
        P.prng_batch_destroy(bt)
        for q, b in zip(reqs, bufs):
            ref = oracle.fill(q["gen"], q["seed"], q["n_streams"], q["n_per"],
                              luxury=q["luxury"]).reshape(-1)[:q["n"]]
            if q["f32"]:
                ref = oracle.to_f32(q["gen"], ref).view(np.uint32)
            np.testing.assert_array_equal(check_pads(b, q["n"]), ref, err_msg=str(q))
    finally:
        for h in handles:
            P.prng_destroy(h)
        for b in bufs:
            b.close()


@pytest.mark.parametrize("gen", inputs.GENS)
def test_large_fill_into_host_equals_device_fill(gen):
    # Full-width launch (every CTA of the bench's u32 fill) into host memory
    # equals the same fill into device memory.
    ns = 8192 if gen == "mt19937" else 131072
    nper = 16 * 624 if gen == "mt19937" else 2048
    lux = 24 if gen == "ranlux" else 0
    b, out = host_buf(ns * nper)
    dev = torch.empty(ns * nper, dtype=torch.int32, device="cuda")
    h1 = P.prng_create(gen, 77, ns, lux)
    h2 = P.prng_create(gen, 77, ns, lux)
    try:
        P.prng_fill_u32(h1, out, nper)
        P.prng_fill_u32(h2, dev, nper)
        torch.cuda.synchronize()
        got = check_pads(b, ns * nper)
        np.testing.assert_array_equal(got, dev.cpu().numpy().view(np.uint32))
        rows = [0, ns // 2, ns - 1]
        for r in rows:
            np.testing.assert_array_equal(got[r * nper:r * nper + 64],
                                          oracle.sample(gen, 77, r, np.arange(64), luxury=lux))
    finally:
        P.prng_destroy(h1)
        P.prng_destroy(h2)
        b.close()
