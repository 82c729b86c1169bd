"""Reference oracle for the six generators -- TEST INFRASTRUCTURE ONLY.

This package wraps ``prng_oracle.c``, a plain single-threaded C implementation
written from the paper's definitions (Demchik, arXiv:1003.1898, Section 3 and
Appendix A).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  The library (``paper_1003_1898_gb300``)
never imports it and shares no code with it.

Every function is pinned to facts outside the oracle (tests/test_oracle_pins.py);
the readings where the paper is silent are listed in the header of
``prng_oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prng_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GGL, XOR128, RANECU, RANMAR, RANLUX, MT19937 = range(6)
NAMES = ("ggl", "xor128", "ranecu", "ranmar", "ranlux", "mt19937")
GEN_IDS = {n: i for i, n in enumerate(NAMES)}
SHIFT = {GGL: 7, RANECU: 7, XOR128: 8, MT19937: 8, RANMAR: 0, RANLUX: 0}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no vector intrinsics)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "prng_oracle.h")))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-I", _HERE])
        os.replace(tmp, _LIB)
    return _LIB


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _f32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
            vp = ctypes.c_void_p
            L.orc_splitmix64.restype = u64
            L.orc_splitmix64.argtypes = [u64]
            L.orc_fill.restype = ctypes.c_int
            L.orc_fill.argtypes = [i32, i32, u64, u64, u32, u64, u64, vp, vp]
            L.orc_sample.restype = ctypes.c_int
            L.orc_sample.argtypes = [i32, i32, u64, u64, vp, u64, vp]
            L.orc_modpow.restype = u64
            L.orc_modpow.argtypes = [u64, u64, u64]
            L.orc_ggl_jump.restype = u32
            L.orc_ggl_jump.argtypes = [u32, u64]
            L.orc_xor128_jump.restype = None
            L.orc_xor128_jump.argtypes = [vp, u64]
            L.orc_mt_jump.restype = None
            L.orc_mt_jump.argtypes = [vp, u64]
            L.orc_mt_charpoly_info.restype = i32
            L.orc_mt_charpoly_info.argtypes = [ctypes.POINTER(i32)]
            L.orc_mt_next.restype = u32
            L.orc_mt_next.argtypes = [vp]
            L.orc_xor128_next.restype = u32
            L.orc_xor128_next.argtypes = [vp]
            L.orc_serial_sample.restype = ctypes.c_int
            L.orc_serial_sample.argtypes = [i32, u64, vp, u64, vp]
            L.orc_serial_fill.restype = ctypes.c_int
            L.orc_serial_fill.argtypes = [i32, u64, u64, vp]
            L.orc_explicit_draws.restype = ctypes.c_int
            L.orc_explicit_draws.argtypes = [i32, i32, vp, u32, u64, vp]
            L.orc_ising_half_sweep.restype = None
            L.orc_ising_half_sweep.argtypes = [i32, vp, vp, i32, u32, u32, i32]
            L.orc_ising_thresholds.restype = None
            L.orc_ising_thresholds.argtypes = [ctypes.c_double, ctypes.POINTER(u32),
                                               ctypes.POINTER(u32)]
            L.orc_ising_energy.restype = ctypes.c_int64
            L.orc_ising_energy.argtypes = [i32, vp]
            L.orc_ising_magnetisation.restype = ctypes.c_int64
            L.orc_ising_magnetisation.argtypes = [i32, vp]
            L.orc_checksum_draws.restype = u64
            L.orc_checksum_draws.argtypes = [i32, i32, u64, u64, u64]
            L.orc_luxury_p.restype = i32
            L.orc_luxury_p.argtypes = [i32]
            L.orc_to_f32.restype = ctypes.c_float
            L.orc_to_f32.argtypes = [i32, u32]
            L.orc_to_f64.restype = ctypes.c_double
            L.orc_to_f64.argtypes = [i32, u32, u32]
            L.orc_fill_f64.restype = ctypes.c_int
            L.orc_fill_f64.argtypes = [i32, i32, u64, u64, u32, u64, u64, vp]
            L.orc_ranecu_comp1.restype = u32
            L.orc_ranecu_comp1.argtypes = [ctypes.POINTER(i32)]
            L.orc_ranecu_comp2.restype = u32
            L.orc_ranecu_comp2.argtypes = [ctypes.POINTER(i32)]
            _lib = L
    return _lib


def gen_id(gen) -> int:
    return GEN_IDS[gen] if isinstance(gen, str) else int(gen)


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(x & (2**64 - 1)))


def luxury_p(luxury: int) -> int:
    return int(lib().orc_luxury_p(luxury))


def fill(gen, seed: int, n_streams: int, n_per: int, *, luxury: int = 0,
         stream0: int = 0, skip: int = 0, want_f32: bool = False):
    """Stream-major draws of streams [stream0, stream0+n_streams), each after
    discarding `skip` draws.  Returns u32 (and f32) arrays of shape
    (n_streams, n_per)."""
    g = gen_id(gen)
    u = np.zeros((n_streams, n_per), dtype=np.uint32)
    f = np.zeros((n_streams, n_per), dtype=np.float32) if want_f32 else None
    rc = lib().orc_fill(g, luxury, seed & (2**64 - 1), stream0, n_streams, skip, n_per,
                        u.ctypes.data, f.ctypes.data if f is not None else None)
    if rc != 0:
        raise ValueError("oracle fill rejected its arguments")
    return (u, f) if want_f32 else u


def fill_f64(gen, seed: int, n_streams: int, n_per: int, *, luxury: int = 0,
             stream0: int = 0, skip: int = 0):
    """Doubles (reading R11) of streams [stream0, stream0+n_streams), each
    made of two consecutive draws; shape (n_streams, n_per)."""
    out = np.zeros((n_streams, n_per), dtype=np.float64)
    rc = lib().orc_fill_f64(gen_id(gen), luxury, seed & (2**64 - 1), stream0, n_streams, skip,
                            n_per, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle fill_f64 rejected its arguments")
    return out


def to_f64(gen, a, b):
    L, g = lib(), gen_id(gen)
    return np.array([L.orc_to_f64(g, int(x), int(y)) for x, y in zip(a, b)], dtype=np.float64)


def sample(gen, seed: int, stream: int, positions, *, luxury: int = 0):
    """Draws at sorted 0-based positions of one stream."""
    pos = np.ascontiguousarray(np.asarray(positions, dtype=np.uint64))
    out = np.zeros(pos.shape[0], dtype=np.uint32)
    rc = lib().orc_sample(gen_id(gen), luxury, seed & (2**64 - 1), stream,
                          pos.ctypes.data, pos.shape[0], out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle sample rejected its arguments")
    return out


def to_f32(gen, v):
    """Exact float conversion, computed in float64 then narrowed."""
    g = gen_id(gen)
    v = np.asarray(v, dtype=np.uint64)
    return ((v >> np.uint64(SHIFT[g])).astype(np.float64) / 16777216.0).astype(np.float32)


def explicit_draws(gen, seeds, n: int, *, luxury: int = 0):
    """n draws of a stream initialised from explicit seeds (see the C header)."""
    sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    out = np.zeros(n, dtype=np.uint32)
    rc = lib().orc_explicit_draws(gen_id(gen), luxury, sd.ctypes.data, sd.shape[0], n,
                                  out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle explicit_draws rejected its arguments")
    return out


def modpow(a: int, e: int, m: int) -> int:
    return int(lib().orc_modpow(a, e, m))


def ggl_jump(x: int, k: int) -> int:
    return int(lib().orc_ggl_jump(x, k))


def xor128_jump(state, k: int):
    """XOR128 state (x, y, z, w) after k steps, by the GF(2) matrix power."""
    s = np.ascontiguousarray(np.asarray(state, dtype=np.uint32).copy())
    lib().orc_xor128_jump(s.ctypes.data, k & (2**64 - 1))
    return s


def xor128_draws_from(state, n: int):
    """n outputs of XOR128 from an explicit state (x, y, z, w)."""
    class _X(ctypes.Structure):
        _fields_ = [("x", ctypes.c_uint32), ("y", ctypes.c_uint32), ("z", ctypes.c_uint32),
                    ("w", ctypes.c_uint32)]
    x, y, z, w = (int(v) for v in state)
    s = _X(x, y, z, w)
    L = lib()
    return np.array([L.orc_xor128_next(ctypes.byref(s)) for _ in range(n)], dtype=np.uint32)


def mt_jump(table, mti: int, k: int):
    """MT19937 table (624 words) k outputs later (mti unchanged)."""
    class _Mt(ctypes.Structure):
        _fields_ = [("mt", ctypes.c_uint32 * 624), ("mti", ctypes.c_int32)]
    s = _Mt()
    s.mt[:] = [int(x) for x in table]
    s.mti = mti
    lib().orc_mt_jump(ctypes.byref(s), k & (2**64 - 1))
    return np.array(s.mt[:], dtype=np.uint32)


def mt_charpoly_info():
    """(degree, number of terms) of MT19937's characteristic polynomial."""
    n = ctypes.c_int32()
    d = lib().orc_mt_charpoly_info(ctypes.byref(n))
    return int(d), int(n.value)


def mt_init_table(seed: int):
    """init_genrand's table for a 32-bit seed (Section 3.7 initialisation)."""
    t = [seed & 0xFFFFFFFF]
    for i in range(1, 624):
        t.append((1812433253 * (t[-1] ^ (t[-1] >> 30)) + i) & 0xFFFFFFFF)
    return np.array(t, dtype=np.uint32)


def mt_draws_from(table, mti: int, n: int, with_state: bool = False):
    """n outputs of MT19937 from an explicit (table, mti) state (and, with
    with_state, the (table, mti) state after them)."""
    class _Mt(ctypes.Structure):
        _fields_ = [("mt", ctypes.c_uint32 * 624), ("mti", ctypes.c_int32)]
    s = _Mt()
    s.mt[:] = [int(x) for x in table]
    s.mti = mti
    L = lib()
    out = np.array([L.orc_mt_next(ctypes.byref(s)) for _ in range(n)], dtype=np.uint32)
    if with_state:
        return out, np.array(s.mt[:], dtype=np.uint32), int(s.mti)
    return out


def serial_sample(gen, x0: int, positions):
    pos = np.ascontiguousarray(np.asarray(positions, dtype=np.uint64))
    out = np.zeros(pos.shape[0], dtype=np.uint32)
    rc = lib().orc_serial_sample(gen_id(gen), x0, pos.ctypes.data, pos.shape[0],
                                 out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle serial_sample rejected its arguments")
    return out


def serial_fill(gen, x0: int, n: int):
    out = np.zeros(n, dtype=np.uint32)
    rc = lib().orc_serial_fill(gen_id(gen), x0, n, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle serial_fill rejected its arguments")
    return out


def checksum_draws(gen, seed: int, stream: int, n: int, *, luxury: int = 0) -> int:
    return int(lib().orc_checksum_draws(gen_id(gen), luxury, seed, stream, n))


def ranecu_components(s1: int, s2: int, n: int):
    """The two MLCG components of RANECU, stepped separately."""
    L = lib()
    a, b = ctypes.c_int32(s1), ctypes.c_int32(s2)
    c1 = np.array([L.orc_ranecu_comp1(ctypes.byref(a)) for _ in range(n)], dtype=np.uint32)
    c2 = np.array([L.orc_ranecu_comp2(ctypes.byref(b)) for _ in range(n)], dtype=np.uint32)
    return c1, c2


# ---------------------------------------------------------------- Ising consumer

ISING_BETA = 0.4406868


def ising_thresholds(beta: float = ISING_BETA):
    t4, t8 = ctypes.c_uint32(), ctypes.c_uint32()
    lib().orc_ising_thresholds(beta, ctypes.byref(t4), ctypes.byref(t8))
    return int(t4.value), int(t8.value)


def ising_half_sweep(spins, draws, gen, colour: int, t4: int, t8: int):
    """In place on an (L, L) int8 array; draws: L*L/2 uint32 (stream-major fill)."""
    L = spins.shape[0]
    assert spins.dtype == np.int8 and spins.flags.c_contiguous
    d = np.ascontiguousarray(draws, dtype=np.uint32).reshape(-1)
    assert d.shape[0] == L * L // 2
    lib().orc_ising_half_sweep(L, spins.ctypes.data, d.ctypes.data, SHIFT[gen_id(gen)], t4, t8,
                               colour)


def ising_energy(spins) -> int:
    return int(lib().orc_ising_energy(spins.shape[0], spins.ctypes.data))


def ising_magnetisation(spins) -> int:
    return int(lib().orc_ising_magnetisation(spins.shape[0], spins.ctypes.data))


def ising_run(gen, seed: int, n_streams: int, L: int, sweeps: int, *, luxury: int = 0,
              beta: float = ISING_BETA, skip: int = 0, spins=None):
    """Cold start (all +1) unless spins is given; each half-sweep takes the
    next L*L/(2 n_streams) draws of every stream of the handle (after `skip`
    draws per stream).  Returns the lattice and the (E, M) after every
    sweep."""
    t4, t8 = ising_thresholds(beta)
    s = np.ones((L, L), dtype=np.int8) if spins is None else spins.copy()
    per = L * L // (2 * n_streams)
    assert per * 2 * n_streams == L * L
    all_draws = fill(gen, seed, n_streams, 2 * sweeps * per, luxury=luxury, skip=skip)
    em = []
    for sw in range(sweeps):
        for colour in (0, 1):
            h = 2 * sw + colour
            ising_half_sweep(s, all_draws[:, h * per:(h + 1) * per], gen, colour, t4, t8)
        em.append((ising_energy(s), ising_magnetisation(s)))
    return s, em
