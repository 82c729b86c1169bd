"""GPU parity: every output of the CUDA library against the CPU oracle.

Integer work, so the bar is bit-exact for u32 and for f32 (every float is
an exact scaling of an integer of at most 24 bits).  All calls go through
the C ABI via the thin Python binding.
"""
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


def lux_of(gen, p=24):
    return p if gen == "ranlux" else 0


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def fill(h, n_streams, n_per, dtype="u32", offset=0):
    """Fill into a fresh buffer (optionally at an element offset)."""
    tdt = torch.float32 if dtype == "f32" else torch.int32
    buf = torch.full((n_streams * n_per + offset + 4,), -7, dtype=tdt, device="cuda")
    view = buf[offset:offset + n_streams * n_per]
    if dtype == "f32":
        P.prng_fill_f32(h, view.data_ptr(), n_per)
    else:
        P.prng_fill_u32(h, view.data_ptr(), n_per)
    torch.cuda.synchronize()
    tail = buf[offset + n_streams * n_per:]
    head = buf[:offset]
    assert torch.all(tail == -7), "write past the end of the output"
    assert torch.all(head == -7), "write before the start of the output"
    return view.reshape(n_streams, n_per) if n_per else view


# ------------------------------------------------------------ small full compare

@pytest.mark.parametrize("gen", inputs.GENS)
def test_small_config_every_element(gen):
    ns, nper = inputs.SMALL["n_streams"], inputs.SMALL["n_per"]
    lux = lux_of(gen)
    ref_u, ref_f = oracle.fill(gen, inputs.SEED_BASE, ns, nper, luxury=lux, want_f32=True)
    h = P.prng_create(gen, inputs.SEED_BASE, ns, lux)
    h2 = P.prng_create(gen, inputs.SEED_BASE, ns, lux)
    try:
        got_u = u32(fill(h, ns, nper))
        got_f = fill(h2, ns, nper, "f32").cpu().numpy()
    finally:
        P.prng_destroy(h)
        P.prng_destroy(h2)
    np.testing.assert_array_equal(got_u, ref_u)
    np.testing.assert_array_equal(got_f.view(np.uint32), ref_f.view(np.uint32))


@pytest.mark.parametrize("p", inputs.LUXURY_LEVELS + inputs.PLANAR_LEVELS)
def test_ranlux_luxury_levels_small(p):
    ns, nper = 96, 1000
    ref = oracle.fill("ranlux", 99, ns, nper, luxury=p)
    h = P.prng_create("ranlux", 99, ns, p)
    try:
        got = u32(fill(h, ns, nper))
    finally:
        P.prng_destroy(h)
    np.testing.assert_array_equal(got, ref)


# ------------------------------------------------------------ ragged shapes and continuation

SHAPES = [(1, 1), (1, 33), (3, 5), (31, 97), (129, 31), (130, 98), (257, 623), (65, 625), (33, 1000)]


@pytest.mark.parametrize("gen", inputs.GENS)
@pytest.mark.parametrize("ns,nper", SHAPES)
def test_ragged_shapes(gen, ns, nper):
    lux = lux_of(gen, 97)
    ref = oracle.fill(gen, 7, ns, nper, luxury=lux, want_f32=True)
    h = P.prng_create(gen, 7, ns, lux)
    h2 = P.prng_create(gen, 7, ns, lux)
    try:
        got = u32(fill(h, ns, nper))
        gotf = fill(h2, ns, nper, "f32").cpu().numpy()
    finally:
        P.prng_destroy(h)
        P.prng_destroy(h2)
    np.testing.assert_array_equal(got, ref[0])
    np.testing.assert_array_equal(gotf.view(np.uint32), ref[1].view(np.uint32))


@pytest.mark.parametrize("gen", inputs.GENS)
def test_successive_fills_continue_each_stream(gen):
    lux = lux_of(gen, 223)
    ns = 70
    pieces = [1, 7, 24, 23, 100, 97, 3, 624, 625, 1, 64, 500]
    total = sum(pieces)
    ref = oracle.fill(gen, 0xABC, ns, total, luxury=lux)
    h = P.prng_create(gen, 0xABC, ns, lux)
    try:
        col = 0
        for i, k in enumerate(pieces):
            dtype = "f32" if i % 3 == 2 else "u32"
            got = fill(h, ns, k, dtype)
            if dtype == "f32":
                want = oracle.to_f32(gen, ref[:, col:col + k])
                np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32), want.view(np.uint32))
            else:
                np.testing.assert_array_equal(u32(got), ref[:, col:col + k])
            col += k
    finally:
        P.prng_destroy(h)


@pytest.mark.parametrize("gen", inputs.GENS)
def test_skip_equals_discarded_fill(gen):
    lux = lux_of(gen, 389)
    ns = 40
    for k, nper in [(1, 10), (23, 50), (24, 24), (97, 130), (1000, 33), (12345, 64)]:
        ref = oracle.fill(gen, 5, ns, nper, luxury=lux, skip=k)
        h = P.prng_create(gen, 5, ns, lux)
        try:
            P.prng_skip(h, k)
            got = u32(fill(h, ns, nper))
        finally:
            P.prng_destroy(h)
        np.testing.assert_array_equal(got, ref, err_msg=f"skip {k}")


def _xor128_seeded(seed, i):
    # Reading R1 for XOR128: s = splitmix64(seed + i), (x, y) = halves of s,
    # (z, w) = halves of splitmix64(s).
    s = oracle.splitmix64(seed + i)
    t = oracle.splitmix64(s)
    return [s & 0xFFFFFFFF, s >> 32, t & 0xFFFFFFFF, t >> 32]


@pytest.mark.parametrize("k", [256, 1000, 65537, 2**40 + 7, 2**64 - 1])
def test_xor128_skip_by_matrix_power(k):
    # Skips of 256 or more run as T^k over GF(2); checked against the
    # oracle's own GF(2) jump of each stream's seeded state.
    ns, nper = 300, 37
    h = P.prng_create("xor128", 11, ns, 0)
    try:
        P.prng_skip(h, k)
        got = u32(fill(h, ns, nper))
    finally:
        P.prng_destroy(h)
    for i in range(ns):
        st = oracle.xor128_jump(_xor128_seeded(11, i), k)
        np.testing.assert_array_equal(got[i], oracle.explicit_draws("xor128", st, nper),
                                      err_msg=f"stream {i}")


def _mt_seeded_table(seed, i):
    # Reading R1 for MT19937: init_genrand(lo32(splitmix64(seed + i))).
    return oracle.mt_init_table(oracle.splitmix64(seed + i) & 0xFFFFFFFF)


@pytest.mark.parametrize("k", [2**20, 2**20 + 1, 10**7 + 3, 2**40 + 7])
@pytest.mark.parametrize("first", [0, 1000])
def test_mt_skip_by_polynomial(k, first):
    # Skips of 2^20 or more move every table k words on by the jump
    # polynomial; checked against the oracle's own jump of each stream's
    # state (after `first` outputs, so from inside a table too).
    ns, nper = 24, 700
    h = P.prng_create("mt19937", 13, ns, 0)
    try:
        if first:
            fill(h, ns, first)
        P.prng_skip(h, k)
        got = u32(fill(h, ns, nper))
    finally:
        P.prng_destroy(h)
    for i in range(ns):
        _, tab, mti = oracle.mt_draws_from(_mt_seeded_table(13, i), 624, first, with_state=True)
        want = oracle.mt_draws_from(oracle.mt_jump(tab, mti, k), mti, nper)
        np.testing.assert_array_equal(got[i], want, err_msg=f"stream {i}")


def test_xor128_skip_matrix_equals_stepping():
    # The same skip on the two sides of the switch: 300 = 255 + 45 steps.
    ns, nper = 129, 20
    a = P.prng_create("xor128", 3, ns, 0)
    b = P.prng_create("xor128", 3, ns, 0)
    try:
        P.prng_skip(a, 300)
        P.prng_skip(b, 255)
        P.prng_skip(b, 45)
        np.testing.assert_array_equal(u32(fill(a, ns, nper)), u32(fill(b, ns, nper)))
    finally:
        P.prng_destroy(a)
        P.prng_destroy(b)


@pytest.mark.parametrize("gen", inputs.GENS)
def test_misaligned_output_scalar_path(gen):
    # Output starting 1 element past a 16-byte boundary forces the scalar
    # copy-out path; n_per not a multiple of 4 as well.
    lux = lux_of(gen, 48)
    ns, nper = 77, 130
    ref = oracle.fill(gen, 3, ns, nper, luxury=lux)
    h = P.prng_create(gen, 3, ns, lux)
    try:
        got = u32(fill(h, ns, nper, offset=1))
    finally:
        P.prng_destroy(h)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("gen", inputs.GENS)
def test_state_checkpoint_roundtrip(gen):
    lux = lux_of(gen, 97)
    ns = 50
    h = P.prng_create(gen, 11, ns, lux)
    try:
        fill(h, ns, 37)                     # leave RANLUX / MT mid-block
        blob = P.prng_get_state(h)
        a = u32(fill(h, ns, 700))
        P.prng_set_state(h, blob)
        b = u32(fill(h, ns, 700))
        np.testing.assert_array_equal(a, b)
        ref = oracle.fill(gen, 11, ns, 700, luxury=lux, skip=37)
        np.testing.assert_array_equal(a, ref)
        bad = bytearray(blob)
        bad[8] ^= 1                          # generator id in the header
        with pytest.raises(P.PrngError):
            P.prng_set_state(h, bytes(bad))
    finally:
        P.prng_destroy(h)


@pytest.mark.parametrize("gen", inputs.GENS)
def test_reseed_restarts_streams(gen):
    lux = lux_of(gen, 24)
    ns = 33
    h = P.prng_create(gen, 1, ns, lux)
    try:
        fill(h, ns, 55)
        P.prng_reseed(h, 2)
        got = u32(fill(h, ns, 200))
    finally:
        P.prng_destroy(h)
    np.testing.assert_array_equal(got, oracle.fill(gen, 2, ns, 200, luxury=lux))


def test_zero_length_fill_is_noop():
    h = P.prng_create("mt19937", 9, 8, 0)
    try:
        P.prng_fill_u32(h, 0, 0)
        got = u32(fill(h, 8, 10))
    finally:
        P.prng_destroy(h)
    np.testing.assert_array_equal(got, oracle.fill("mt19937", 9, 8, 10))


def test_fill_rejects_bad_sizes_before_launching():
    # Host validation: sizes whose element count overflows 64 bits and
    # misaligned outputs are rejected with nothing launched; the stream is
    # unchanged afterwards.
    h = P.prng_create("xor128", 5, 8, 0)
    buf = torch.empty(64, dtype=torch.int32, device="cuda")
    try:
        for fn, n, ptr, code in [(P.prng_fill_u32, 2**62, buf.data_ptr(), -3),
                                 (P.prng_fill_f32, 2**61 + 1, buf.data_ptr(), -3),
                                 (P.prng_fill_f64, 2**63 + 1, buf.data_ptr(), -3),
                                 (P.prng_fill_u32, 4, buf.data_ptr() + 2, -3),
                                 (P.prng_fill_f64, 4, buf.data_ptr() + 4, -3),
                                 (P.prng_fill_u32, 4, 0, -4)]:
            with pytest.raises(P.PrngError) as err:
                fn(h, ptr, n)
            assert err.value.code == code, (fn.__name__, n)
        got = u32(fill(h, 8, 10))
    finally:
        P.prng_destroy(h)
    np.testing.assert_array_equal(got, oracle.fill("xor128", 5, 8, 10))


# ------------------------------------------------------------ jump-ahead

@pytest.mark.parametrize("gen", ["ggl", "ranecu", "xor128", "mt19937"])
@pytest.mark.parametrize("n,chunks", [(1, 1), (1000, 7), (100003, 37), (65536, 512), (50000, 1)])
def test_jump_fill_small_every_element(gen, n, chunks):
    x0 = inputs.JUMP_X0[gen]
    ref = oracle.serial_fill(gen, x0, n)
    out = torch.full((n + 4,), -7, dtype=torch.int32, device="cuda")
    P.prng_fill_jump_u32(gen, x0, n, chunks, out.data_ptr())
    outf = torch.full((n,), -7.0, dtype=torch.float32, device="cuda")
    P.prng_fill_jump_f32(gen, x0, n, chunks, outf.data_ptr())
    torch.cuda.synchronize()
    got = u32(out)
    np.testing.assert_array_equal(got[:n], ref)
    assert np.all(got[n:] == np.uint32(2**32 - 7))
    np.testing.assert_array_equal(outf.cpu().numpy().view(np.uint32),
                                  oracle.to_f32(gen, ref).view(np.uint32))


@pytest.mark.parametrize("gen", ["ggl", "ranecu", "xor128", "mt19937"])
def test_jump_fill_other_start(gen):
    x0 = {"ggl": 123456789, "ranecu": 987654 | (13579 << 32), "xor128": 0, "mt19937": 4357}[gen]
    n = 77777
    out = torch.empty((n,), dtype=torch.int32, device="cuda")
    P.prng_fill_jump_u32(gen, x0, n, 100, out.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(u32(out), oracle.serial_fill(gen, x0, n))


def _jump_ref(gen, x0, first, n):
    """Draws first+1 .. first+n of the single sequence from x0, by the
    oracle: its start moved `first` draws on with the oracle's own jump
    (GGL, XOR128, MT19937) or modular power (RANECU, per component), then
    stepped serially."""
    if gen == "ggl":
        return oracle.serial_fill("ggl", oracle.ggl_jump(x0, first), n)
    if gen == "ranecu":
        s1 = oracle.modpow(40014, first, 2147483563) * (x0 & 0xFFFFFFFF) % 2147483563
        s2 = oracle.modpow(40692, first, 2147483399) * (x0 >> 32) % 2147483399
        return oracle.serial_fill("ranecu", s1 | (s2 << 32), n)
    if gen == "xor128":
        t = oracle.splitmix64(x0)
        st = [x0 & 0xFFFFFFFF, (x0 >> 32) & 0xFFFFFFFF, t & 0xFFFFFFFF, t >> 32]
        return oracle.xor128_draws_from(oracle.xor128_jump(st, first), n)
    return oracle.mt_draws_from(oracle.mt_jump(oracle.mt_init_table(x0), 624, first), 624, n)


@pytest.mark.parametrize("gen", ["ggl", "ranecu", "xor128", "mt19937"])
@pytest.mark.parametrize("first", [0, 1, 123457, 2**40 + 3, 2**63 + 5])
def test_jump_fill_at_offset(gen, first):
    x0 = inputs.JUMP_X0[gen]
    n, chunks = 20011, 37
    out = torch.full((n + 4,), -7, dtype=torch.int32, device="cuda")
    P.prng_fill_jump_at_u32(gen, x0, first, n, chunks, out.data_ptr())
    torch.cuda.synchronize()
    got = u32(out)
    np.testing.assert_array_equal(got[:n], _jump_ref(gen, x0, first, n))
    assert np.all(got[n:] == np.uint32(2**32 - 7)), "write past the end"
    if first < 10**6:   # small offsets: the plain serial oracle directly
        np.testing.assert_array_equal(got[:n], oracle.serial_sample(gen, x0, first + np.arange(n)))


@pytest.mark.parametrize("gen", ["ggl", "ranecu", "xor128", "mt19937"])
def test_jump_fill_at_ranges_tile_one_sequence(gen):
    # Two ranks' ranges [0, n) and [n, 2n), as f32, equal the one fill of 2n.
    x0 = inputs.JUMP_X0[gen]
    n = 30000
    whole = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    P.prng_fill_jump_f32(gen, x0, 2 * n, 64, whole)
    parts = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    P.prng_fill_jump_at_f32(gen, x0, 0, n, 32, parts[:n])
    P.prng_fill_jump_at_f32(gen, x0, n, n, 32, parts[n:])
    torch.cuda.synchronize()
    assert torch.equal(whole.view(torch.int32), parts.view(torch.int32))
    ref = oracle.to_f32(gen, oracle.serial_fill(gen, x0, 2 * n))
    np.testing.assert_array_equal(parts.cpu().numpy().view(np.uint32), ref.view(np.uint32))


# ------------------------------------------------------------ full sizes (sampled)

def _sampled_rows_check(gen, lux, ns, nper, n_rows_checked, dtype="u32"):
    h = P.prng_create(gen, inputs.SEED_BASE, ns, lux)
    try:
        tdt = torch.float32 if dtype == "f32" else torch.int32
        out = torch.empty((ns, nper), dtype=tdt, device="cuda")
        if dtype == "f32":
            P.prng_fill_f32(h, out, nper)
        else:
            P.prng_fill_u32(h, out, nper)
        torch.cuda.synchronize()
        rows = inputs.sample_rows(ns, n_rows_checked)
        got = out[torch.as_tensor(rows, device="cuda")].cpu().numpy()
        for i, r in enumerate(rows):
            ref = oracle.fill(gen, inputs.SEED_BASE, 1, nper, luxury=lux, stream0=int(r))[0]
            if dtype == "f32":
                np.testing.assert_array_equal(got[i].view(np.uint32),
                                              oracle.to_f32(gen, ref).view(np.uint32))
            else:
                np.testing.assert_array_equal(got[i].view(np.uint32), ref, err_msg=f"row {r}")
        # properties over every element: range of the integer / float outputs
        if dtype == "f32":
            assert float(out.min()) >= 0.0 and float(out.max()) < 1.0
            scaled = out.double() * 2.0**24
            assert bool(torch.all(scaled == torch.floor(scaled)))
        del out
    finally:
        P.prng_destroy(h)


@pytest.mark.parametrize("gen", ["ggl", "xor128", "ranecu", "ranmar", "ranlux"])
@pytest.mark.parametrize("dtype", ["u32", "f32"])
def test_roofline_config_sampled(gen, dtype):
    cfg = inputs.ROOFLINE
    _sampled_rows_check(gen, lux_of(gen, 24), cfg["n_streams"], cfg["n_per"], 24, dtype)


@pytest.mark.parametrize("dtype", ["u32", "f32"])
def test_roofline_config_mt_sampled(dtype):
    cfg = inputs.ROOFLINE_MT
    _sampled_rows_check("mt19937", 0, cfg["n_streams"], cfg["n_per"], 8, dtype)


@pytest.mark.parametrize("p", inputs.LUXURY_LEVELS + inputs.PLANAR_LEVELS)
def test_luxury_sweep_config_sampled(p):
    cfg = inputs.LUX_SWEEP
    _sampled_rows_check("ranlux", p, cfg["n_streams"], cfg["n_per"], 8, "f32")


@pytest.mark.parametrize("gen", ["ggl", "ranecu", "xor128", "mt19937"])
def test_jump_full_size_sampled(gen):
    n, chunks = inputs.JUMP["n"], inputs.JUMP["n_chunks"]
    if gen == "mt19937":
        chunks = inputs.ROOFLINE_MT["n_streams"]     # one warp per chunk, as the bulk fill
    x0 = inputs.JUMP_X0[gen]
    out = torch.empty((n,), dtype=torch.int32, device="cuda")
    P.prng_fill_jump_u32(gen, x0, n, chunks, out.data_ptr())
    torch.cuda.synchronize()
    pos = inputs.jump_offsets(n, chunks)
    got = out[torch.as_tensor(pos.astype(np.int64), device="cuda")].cpu().numpy().view(np.uint32)
    ref = oracle.serial_sample(gen, x0, pos)
    np.testing.assert_array_equal(got, ref)
    if gen == "ggl":
        assert int(got[np.searchsorted(pos, 9999)]) == 1043618065
    if gen == "mt19937":
        assert int(got[np.searchsorted(pos, 9999)]) == 4123659995
    del out


# ------------------------------------------------------------ doubles from pairs

def fill_f64(h, n_streams, n_per, offset=0):
    buf = torch.full((n_streams * n_per + offset + 2,), -7.0, dtype=torch.float64, device="cuda")
    view = buf[offset:offset + n_streams * n_per]
    P.prng_fill_f64(h, view.data_ptr(), n_per)
    torch.cuda.synchronize()
    assert torch.all(buf[offset + n_streams * n_per:] == -7.0), "write past the end"
    assert torch.all(buf[:offset] == -7.0), "write before the start"
    return view.reshape(n_streams, n_per).cpu().numpy()


@pytest.mark.parametrize("gen", inputs.GENS)
@pytest.mark.parametrize("ns,nper", [(1, 1), (130, 333), (257, 1000), (33, 4096)])
def test_f64_every_element(gen, ns, nper):
    lux = lux_of(gen, 223)
    ref = oracle.fill_f64(gen, 21, ns, nper, luxury=lux)
    h = P.prng_create(gen, 21, ns, lux)
    try:
        got = fill_f64(h, ns, nper)
    finally:
        P.prng_destroy(h)
    np.testing.assert_array_equal(got.view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("gen", inputs.GENS)
def test_f64_continues_u32_and_f32_fills(gen):
    # u32 (even count), f64, f32, f64 on one handle = the oracle stream cut there.
    lux = lux_of(gen, 97)
    ns = 70
    h = P.prng_create(gen, 8, ns, lux)
    try:
        a = u32(fill(h, ns, 50))
        b = fill_f64(h, ns, 61)
        c = fill(h, ns, 30, "f32").cpu().numpy()
        d = fill_f64(h, ns, 700, offset=1)          # 8- but not 16-byte aligned
    finally:
        P.prng_destroy(h)
    np.testing.assert_array_equal(a, oracle.fill(gen, 8, ns, 50, luxury=lux))
    np.testing.assert_array_equal(b.view(np.uint64),
                                  oracle.fill_f64(gen, 8, ns, 61, luxury=lux, skip=50).view(np.uint64))
    _, cf = oracle.fill(gen, 8, ns, 30, luxury=lux, skip=172, want_f32=True)
    np.testing.assert_array_equal(c.view(np.uint32), cf.view(np.uint32))
    np.testing.assert_array_equal(d.view(np.uint64),
                                  oracle.fill_f64(gen, 8, ns, 700, luxury=lux, skip=202).view(np.uint64))


@pytest.mark.parametrize("gen", ["ranlux", "mt19937"])
def test_f64_needs_even_position(gen):
    lux = lux_of(gen, 24)
    h = P.prng_create(gen, 5, 40, lux)
    try:
        fill(h, 40, 7)                                   # odd count: odd position
        out = torch.full((40 * 10,), -7.0, dtype=torch.float64, device="cuda")
        with pytest.raises(P.PrngError) as err:
            P.prng_fill_f64(h, out.data_ptr(), 10)
        assert err.value.code == -11
        torch.cuda.synchronize()
        assert torch.all(out == -7.0)
        P.prng_skip(h, 1)
        got = fill_f64(h, 40, 10)
    finally:
        P.prng_destroy(h)
    np.testing.assert_array_equal(got.view(np.uint64),
                                  oracle.fill_f64(gen, 5, 40, 10, luxury=lux, skip=8).view(np.uint64))


@pytest.mark.parametrize("p", inputs.LUXURY_LEVELS)
def test_f64_ranlux_levels_from_even_positions(p):
    ns = 65
    h = P.prng_create("ranlux", 31, ns, p)
    try:
        fill(h, ns, 10)                                  # position 10 of the first block
        got = fill_f64(h, ns, 101)
    finally:
        P.prng_destroy(h)
    np.testing.assert_array_equal(got.view(np.uint64),
                                  oracle.fill_f64("ranlux", 31, ns, 101, luxury=p, skip=10).view(np.uint64))


@pytest.mark.parametrize("gen", ["ggl", "ranmar", "mt19937"])
def test_f64_full_size_sampled(gen):
    ns, nper = (inputs.ROOFLINE_MT["n_streams"], inputs.ROOFLINE_MT["n_per"] // 2) if gen == "mt19937" \
        else (inputs.ROOFLINE["n_streams"], inputs.ROOFLINE["n_per"] // 2)
    h = P.prng_create(gen, inputs.SEED_BASE, ns, 0)
    try:
        out = torch.empty((ns, nper), dtype=torch.float64, device="cuda")
        P.prng_fill_f64(h, out.data_ptr(), nper)
        torch.cuda.synchronize()
        rows = inputs.sample_rows(ns, 6)
        got = out[torch.as_tensor(rows, device="cuda")].cpu().numpy()
        for i, r in enumerate(rows):
            ref = oracle.fill_f64(gen, inputs.SEED_BASE, 1, nper, stream0=int(r))[0]
            np.testing.assert_array_equal(got[i].view(np.uint64), ref.view(np.uint64), err_msg=f"row {r}")
        assert float(out.min()) >= 0.0 and float(out.max()) < 1.0
    finally:
        P.prng_destroy(h)
        del out
