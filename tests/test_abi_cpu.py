"""The C ABI without a GPU: the library loads, exports every entry point
declared in include/prng.h, and rejects bad arguments on the host before
any CUDA call."""
import ctypes
import os
import re

import pytest

import paper_1003_1898_gb300 as P
from paper_1003_1898_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return P.lib()


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(prng_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


def test_create_rejects_bad_arguments(L):
    h = ctypes.c_void_p()
    assert L.prng_create(ctypes.byref(h), 6, 1, 10, 0) == -1          # generator
    assert L.prng_create(ctypes.byref(h), -1, 1, 10, 0) == -1
    assert L.prng_create(ctypes.byref(h), P.RANLUX, 1, 10, 5) == -2   # luxury
    assert L.prng_create(ctypes.byref(h), P.RANLUX, 1, 10, 100) == -2
    assert L.prng_create(ctypes.byref(h), P.GGL, 1, 0, 0) == -3       # no streams
    assert L.prng_create(None, P.GGL, 1, 10, 0) == -4
    assert h.value is None


def test_jump_rejects_bad_arguments(L):
    buf = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    assert L.prng_fill_jump_u32(P.RANMAR, 1, 10, 1, buf, None) == -7
    assert L.prng_fill_jump_u32(P.RANLUX, 1, 10, 1, buf, None) == -7
    assert L.prng_fill_jump_u32(P.MT19937, 2**32, 10, 1, buf, None) == -9    # MT: 32-bit seed
    assert L.prng_fill_jump_u32(P.XOR128, 1, 10, 0, buf, None) == -3      # XOR128: no chunks
    assert L.prng_fill_jump_u32(P.XOR128, 1, 10, 1, None, None) == -4
    assert L.prng_fill_jump_u32(9, 1, 10, 1, buf, None) == -1
    assert L.prng_fill_jump_u32(P.GGL, 0, 10, 1, buf, None) == -9
    assert L.prng_fill_jump_u32(P.GGL, 2**31 - 1, 10, 1, buf, None) == -9
    assert L.prng_fill_jump_u32(P.RANECU, 1, 10, 1, buf, None) == -9      # s2 = 0
    assert L.prng_fill_jump_u32(P.RANECU, 2147483563 | (1 << 32), 10, 1, buf, None) == -9
    assert L.prng_fill_jump_u32(P.GGL, 1, 10, 0, buf, None) == -3
    assert L.prng_fill_jump_u32(P.GGL, 1, 10, 1, None, None) == -4
    assert L.prng_fill_jump_u32(P.GGL, 1, 0, 1, None, None) == 0          # empty: no-op
    assert L.prng_fill_jump_at_u32(P.GGL, 1, 2**64 - 5, 10, 1, buf, None) == -3   # first + n overflows
    assert L.prng_fill_jump_at_u32(P.RANMAR, 1, 0, 10, 1, buf, None) == -7
    assert L.prng_fill_jump_at_u32(P.MT19937, 2**32, 5, 10, 1, buf, None) == -9
    assert L.prng_fill_jump_at_u32(P.GGL, 0, 5, 10, 1, buf, None) == -9
    assert L.prng_fill_jump_at_f32(P.XOR128, 1, 5, 10, 1, None, None) == -4
    assert L.prng_fill_jump_at_u32(P.GGL, 1, 5, 0, 1, None, None) == 0       # empty: no-op


def test_null_handles(L):
    assert L.prng_fill_u32(None, None, 10, None) == -4
    assert L.prng_skip(None, 3, None) == -4
    assert L.prng_info(None, None, None, None, None) == -4
    n = ctypes.c_size_t()
    assert L.prng_get_state(None, None, ctypes.byref(n)) == -4
    L.prng_destroy(None)


def test_host_alloc_rejects_bad_arguments(L):
    p = ctypes.c_void_p()
    assert L.prng_host_alloc(None, 64) == -4
    assert L.prng_host_alloc(ctypes.byref(p), 0) == -3
    assert p.value is None
    assert L.prng_host_free(None) == 0


def test_strerror_names_every_code(L):
    for code in range(0, -12, -1):
        s = P.prng_strerror(code)
        assert s and s != "unknown error code"
    assert P.prng_strerror(-99) == "unknown error code"


def test_batch_create_rejects_bad_arguments(L):
    b = ctypes.c_void_p()
    assert L.prng_batch_create(None, None, 1) == -4
    assert L.prng_batch_create(ctypes.byref(b), None, 0) == -3
    assert L.prng_batch_create(ctypes.byref(b), None, 3) == -4
    reqs = (P.PrngFillReq * 1)()          # st = NULL
    assert L.prng_batch_create(ctypes.byref(b), reqs, 1) == -4
    assert L.prng_batch_launch(None, None) == -4
    assert L.prng_batch_info(None, None, None, None) == -4
    L.prng_batch_destroy(None)
