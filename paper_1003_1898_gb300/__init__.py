"""paper_1003_1898_gb300 -- Python binding of libprng (GB300 uniform PRNGs).

Argument marshalling only: every function forwards to the C entry point of
the same name in ``libprng.so`` (declared in ``include/prng.h``); every draw
is produced by the library's CUDA kernels.  PyTorch is used for device
memory and the current CUDA stream.  If the shared library has not been
built, ``lib()`` raises -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libprng.so")

GGL, XOR128, RANECU, RANMAR, RANLUX, MT19937 = range(6)
GEN_NAMES = ("ggl", "xor128", "ranecu", "ranmar", "ranlux", "mt19937")
GEN_IDS = {n: i for i, n in enumerate(GEN_NAMES)}
LUXURY_P = (24, 48, 97, 223, 389)
PLANAR_P = (48, 120, 240, 408)          # Section 3.6 planar scheme: 24, 96, 216, 384 discarded
STATE_WORDS = (1, 4, 2, 98, 25, 624)

_lib = None


class PrngIsingReq(ctypes.Structure):
    """struct prng_ising_req (include/prng.h)."""
    _fields_ = [("d_spins", ctypes.c_void_p), ("d_draws", ctypes.c_void_p), ("L", ctypes.c_uint32),
                ("colour", ctypes.c_uint32), ("shift", ctypes.c_uint32), ("t4", ctypes.c_uint32),
                ("t8", ctypes.c_uint32), ("per", ctypes.c_uint32), ("pitch", ctypes.c_uint32)]


class PrngFillReq(ctypes.Structure):
    """struct prng_fill_req (include/prng.h)."""
    _fields_ = [("st", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
                ("n_per_stream", ctypes.c_uint64), ("n_valid", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("f32", ctypes.c_uint32), ("reseed", ctypes.c_uint32)]


def _np_dtype(struct):
    """numpy structured dtype with the exact field offsets and size of a
    ctypes struct, so arrays of it can be handed to the library as is."""
    import numpy as np
    fmt = {ctypes.c_void_p: "<u8", ctypes.c_uint64: "<u8", ctypes.c_uint32: "<u4"}
    names = [n for n, _ in struct._fields_]
    return np.dtype({"names": names, "formats": [fmt[t] for _, t in struct._fields_],
                     "offsets": [getattr(struct, n).offset for n in names],
                     "itemsize": ctypes.sizeof(struct)})


FILL_REQ_DTYPE = _np_dtype(PrngFillReq)
ISING_REQ_DTYPE = _np_dtype(PrngIsingReq)


def _struct_rows(rows, dtype, struct):
    """(pointer, count) of a numpy array of `dtype` rows, passed as is."""
    import numpy as np
    arr = np.ascontiguousarray(rows)
    if arr.dtype != dtype:
        raise TypeError(f"expected rows of {dtype}")
    return arr, arr.ctypes.data_as(ctypes.POINTER(struct)), arr.shape[0]


class PrngError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {prng_strerror(code)} (code {code})")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libprng.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libprng.so is not built ({LIB_PATH}); run "
                           "paper_1003_1898_gb300.build.build() first")
    L = ctypes.CDLL(LIB_PATH)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
    sig = {
        "prng_create": ([ctypes.POINTER(vp), ctypes.c_int, u64, u32, u32], ctypes.c_int),
        "prng_reseed": ([vp, u64, vp], ctypes.c_int),
        "prng_fill_u32": ([vp, vp, u64, vp], ctypes.c_int),
        "prng_fill_f32": ([vp, vp, u64, vp], ctypes.c_int),
        "prng_fill_f64": ([vp, vp, u64, vp], ctypes.c_int),
        "prng_skip": ([vp, u64, vp], ctypes.c_int),
        "prng_get_state": ([vp, vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "prng_set_state": ([vp, vp, ctypes.c_size_t], ctypes.c_int),
        "prng_fill_jump_u32": ([ctypes.c_int, u64, u64, u32, vp, vp], ctypes.c_int),
        "prng_fill_jump_f32": ([ctypes.c_int, u64, u64, u32, vp, vp], ctypes.c_int),
        "prng_fill_jump_at_u32": ([ctypes.c_int, u64, u64, u64, u32, vp, vp], ctypes.c_int),
        "prng_fill_jump_at_f32": ([ctypes.c_int, u64, u64, u64, u32, vp, vp], ctypes.c_int),
        "prng_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(u32),
                       ctypes.POINTER(u64)], ctypes.c_int),
        "prng_set_tile": ([ctypes.c_int, u32, u32, u32, u32], ctypes.c_int),
        "prng_get_tile": ([ctypes.c_int, u32, ctypes.POINTER(u32), ctypes.POINTER(u32),
                           ctypes.POINTER(u32)], ctypes.c_int),
        "prng_batch_create": ([ctypes.POINTER(vp), ctypes.POINTER(PrngFillReq), u32], ctypes.c_int),
        "prng_batch_launch": ([vp, vp], ctypes.c_int),
        "prng_batch_info": ([vp, ctypes.POINTER(u32), ctypes.POINTER(u64), ctypes.POINTER(u64)],
                            ctypes.c_int),
        "prng_batch_destroy": ([vp], None),
        "prng_batch_fill_noalloc": ([ctypes.POINTER(PrngFillReq), u32, vp], ctypes.c_int),
        "prng_batcher_create": ([ctypes.POINTER(vp), u32, u64], ctypes.c_int),
        "prng_batcher_launch": ([vp, ctypes.POINTER(PrngFillReq), u32, vp], ctypes.c_int),
        "prng_batcher_destroy": ([vp], None),
        "prng_ising_half_sweep": ([ctypes.POINTER(PrngIsingReq), u32, vp], ctypes.c_int),
        "prng_ising_fused": ([vp, vp, u32, u32, u32, u32, vp], ctypes.c_int),
        "prng_ising_thresholds": ([ctypes.c_double, ctypes.POINTER(u32), ctypes.POINTER(u32)],
                                  ctypes.c_int),
        "prng_float_shift": ([ctypes.c_int, ctypes.POINTER(u32)], ctypes.c_int),
        "prng_calib_swb": ([u32, u32, u32, vp, u64, ctypes.POINTER(u64), vp], ctypes.c_int),
        "prng_host_alloc": ([ctypes.POINTER(vp), ctypes.c_size_t], ctypes.c_int),
        "prng_host_free": ([vp], ctypes.c_int),
        "prng_destroy": ([vp], None),
        "prng_strerror": ([ctypes.c_int], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _gen(gen) -> int:
    return GEN_IDS[gen] if isinstance(gen, str) else int(gen)


def _ptr(x) -> int:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()   # torch tensor


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def _check(rc: int, what: str):
    if rc != 0:
        raise PrngError(rc, what)


def prng_strerror(code: int) -> str:
    return lib().prng_strerror(code).decode()


def prng_create(gen, seed: int, n_streams: int, luxury: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().prng_create(ctypes.byref(h), _gen(gen), seed & (2**64 - 1), n_streams, luxury),
           "prng_create")
    return h


def prng_reseed(h, seed: int, stream=None):
    _check(lib().prng_reseed(h, seed & (2**64 - 1), _stream(stream)), "prng_reseed")


def prng_fill_u32(h, out, n_per_stream: int, stream=None):
    _check(lib().prng_fill_u32(h, _ptr(out), n_per_stream, _stream(stream)), "prng_fill_u32")


def prng_fill_f32(h, out, n_per_stream: int, stream=None):
    _check(lib().prng_fill_f32(h, _ptr(out), n_per_stream, _stream(stream)), "prng_fill_f32")


def prng_fill_f64(h, out, n_per_stream: int, stream=None):
    """Doubles from pairs of draws: each stream advances by 2 n_per_stream."""
    _check(lib().prng_fill_f64(h, _ptr(out), n_per_stream, _stream(stream)), "prng_fill_f64")


def prng_skip(h, k: int, stream=None):
    _check(lib().prng_skip(h, k, _stream(stream)), "prng_skip")


def prng_get_state(h) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().prng_get_state(h, None, ctypes.byref(n)), "prng_get_state")
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().prng_get_state(h, buf, ctypes.byref(n)), "prng_get_state")
    return buf.raw[:n.value]


def prng_set_state(h, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().prng_set_state(h, buf, len(blob)), "prng_set_state")


def prng_fill_jump_u32(gen, x0: int, n: int, n_chunks: int, out, stream=None):
    _check(lib().prng_fill_jump_u32(_gen(gen), x0, n, n_chunks, _ptr(out), _stream(stream)),
           "prng_fill_jump_u32")


def prng_fill_jump_f32(gen, x0: int, n: int, n_chunks: int, out, stream=None):
    _check(lib().prng_fill_jump_f32(_gen(gen), x0, n, n_chunks, _ptr(out), _stream(stream)),
           "prng_fill_jump_f32")


def prng_fill_jump_at_u32(gen, x0: int, first: int, n: int, n_chunks: int, out, stream=None):
    _check(lib().prng_fill_jump_at_u32(_gen(gen), x0, first, n, n_chunks, _ptr(out), _stream(stream)),
           "prng_fill_jump_at_u32")


def prng_fill_jump_at_f32(gen, x0: int, first: int, n: int, n_chunks: int, out, stream=None):
    _check(lib().prng_fill_jump_at_f32(_gen(gen), x0, first, n, n_chunks, _ptr(out), _stream(stream)),
           "prng_fill_jump_at_f32")


def prng_info(h) -> dict:
    g, p = ctypes.c_int32(), ctypes.c_int32()
    n, b = ctypes.c_uint32(), ctypes.c_uint64()
    _check(lib().prng_info(h, ctypes.byref(g), ctypes.byref(p), ctypes.byref(n), ctypes.byref(b)),
           "prng_info")
    return {"gen": g.value, "p": p.value, "n_streams": n.value, "state_bytes": b.value}


def prng_set_tile(gen, luxury: int, threads: int, cols: int, stages: int):
    _check(lib().prng_set_tile(_gen(gen), luxury, threads, cols, stages), "prng_set_tile")


def prng_get_tile(gen, luxury: int = 0):
    t, c, s = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().prng_get_tile(_gen(gen), luxury, ctypes.byref(t), ctypes.byref(c), ctypes.byref(s)),
           "prng_get_tile")
    return (t.value, c.value, s.value)


def _fill_req_array(reqs):
    reqs = list(reqs)
    arr = (PrngFillReq * max(1, len(reqs)))()
    for i, r in enumerate(reqs):
        st = r["st"]
        arr[i].st = st.value if isinstance(st, ctypes.c_void_p) else st
        arr[i].d_out = _ptr(r["d_out"])
        arr[i].n_per_stream = r["n_per_stream"]
        arr[i].n_valid = r.get("n_valid", 0)
        arr[i].seed = r.get("seed", 0) & (2**64 - 1)
        arr[i].f32 = 1 if r.get("f32", False) else 0
        arr[i].reseed = 1 if r.get("reseed", False) else 0
    return arr, len(reqs)


def prng_batch_create(reqs) -> ctypes.c_void_p:
    """reqs: iterable of dicts with keys st, d_out, n_per_stream and optional
    n_valid, seed, f32, reseed."""
    arr, n = _fill_req_array(reqs)
    b = ctypes.c_void_p()
    _check(lib().prng_batch_create(ctypes.byref(b), arr, n), "prng_batch_create")
    return b


def prng_batch_fill_noalloc(reqs, stream=None):
    """The batched fill through the library's fixed scratch (allocates
    nothing); same request dicts as prng_batch_create."""
    arr, n = _fill_req_array(reqs)
    _check(lib().prng_batch_fill_noalloc(arr, n, _stream(stream)), "prng_batch_fill_noalloc")


def prng_batch_launch(b, stream=None):
    _check(lib().prng_batch_launch(b, _stream(stream)), "prng_batch_launch")


def prng_batch_info(b) -> dict:
    n, it, num = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().prng_batch_info(b, ctypes.byref(n), ctypes.byref(it), ctypes.byref(num)),
           "prng_batch_info")
    return {"requests": n.value, "items": it.value, "numbers": num.value}


def prng_batch_destroy(b):
    lib().prng_batch_destroy(b)


def prng_batcher_create(max_requests: int, max_items: int) -> ctypes.c_void_p:
    b = ctypes.c_void_p()
    _check(lib().prng_batcher_create(ctypes.byref(b), max_requests, max_items),
           "prng_batcher_create")
    return b


def prng_batcher_launch(b, reqs, stream=None):
    """reqs: dicts as for prng_batch_create, or a numpy array of
    FILL_REQ_DTYPE rows (passed to the library without conversion)."""
    if hasattr(reqs, "dtype"):
        keep, arr, n = _struct_rows(reqs, FILL_REQ_DTYPE, PrngFillReq)
    else:
        arr, n = _fill_req_array(reqs)
    _check(lib().prng_batcher_launch(b, arr, n, _stream(stream)), "prng_batcher_launch")


def prng_batcher_destroy(b):
    lib().prng_batcher_destroy(b)


def prng_float_shift(gen) -> int:
    """The generator's float shift: f32 = (v >> sh) 2^-24, and v >> sh is
    the Ising acceptance value."""
    sh = ctypes.c_uint32()
    _check(lib().prng_float_shift(_gen(gen), ctypes.byref(sh)), "prng_float_shift")
    return sh.value


def prng_calib_swb(chains: int, warps_per_sm: int, iters: int, sink, stream=None) -> int:
    """Launch the subtract-with-borrow calibration kernel; returns the integer
    instructions it executes (time the launch with events)."""
    ops = ctypes.c_uint64()
    _check(lib().prng_calib_swb(chains, warps_per_sm, iters, _ptr(sink), sink.numel(),
                                ctypes.byref(ops), _stream(stream)), "prng_calib_swb")
    return ops.value


def prng_ising_thresholds(beta: float):
    t4, t8 = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().prng_ising_thresholds(beta, ctypes.byref(t4), ctypes.byref(t8)),
           "prng_ising_thresholds")
    return t4.value, t8.value


def prng_ising_half_sweep(reqs, stream=None):
    """reqs: iterable of dicts with d_spins, d_draws, L, colour, gen (or
    shift), t4, t8, and optionally per and pitch (the draws of the
    half-sweep as per-word columns of rows `pitch` words apart); d_draws may
    be an integer device address.  A numpy array of ISING_REQ_DTYPE rows is
    passed to the library without conversion."""
    if hasattr(reqs, "dtype"):
        keep, arr, n = _struct_rows(reqs, ISING_REQ_DTYPE, PrngIsingReq)
        _check(lib().prng_ising_half_sweep(arr, n, _stream(stream)), "prng_ising_half_sweep")
        return
    reqs = list(reqs)
    arr = (PrngIsingReq * max(1, len(reqs)))()
    for i, r in enumerate(reqs):
        arr[i].d_spins = _ptr(r["d_spins"])
        arr[i].d_draws = _ptr(r["d_draws"])
        arr[i].L = r["L"]
        arr[i].colour = r["colour"]
        arr[i].shift = r["shift"] if "shift" in r else prng_float_shift(r["gen"])
        arr[i].t4 = r["t4"]
        arr[i].t8 = r["t8"]
        arr[i].per = r.get("per", 0)
        arr[i].pitch = r.get("pitch", 0)
    _check(lib().prng_ising_half_sweep(arr, len(reqs), _stream(stream)), "prng_ising_half_sweep")


def prng_ising_fused(h, spins, L: int, colour: int, t4: int, t8: int, stream=None):
    """One half-sweep of the lattice consuming the handle's next L*L/2 draws
    where they are made (no draw buffer)."""
    _check(lib().prng_ising_fused(h, _ptr(spins), L, colour, t4, t8, _stream(stream)),
           "prng_ising_fused")


def prng_host_alloc(nbytes: int) -> int:
    """Page-locked host memory mapped at the same device address: fills given
    this pointer store their numbers straight into host memory."""
    p = ctypes.c_void_p()
    _check(lib().prng_host_alloc(ctypes.byref(p), nbytes), "prng_host_alloc")
    return p.value


def prng_host_free(ptr):
    _check(lib().prng_host_free(ptr), "prng_host_free")


class HostBuffer:
    """Host output buffer from prng_host_alloc: pass ``.ptr`` (or the buffer
    itself) as a fill's output; read it through ``.numpy(dtype)`` after the
    fill's stream has been synchronised."""

    def __init__(self, nbytes: int):
        self.nbytes = int(nbytes)
        self.ptr = prng_host_alloc(self.nbytes)

    def data_ptr(self) -> int:
        return self.ptr

    def numpy(self, dtype="uint32", count: int | None = None):
        import numpy as np
        dt = np.dtype(dtype)
        n = self.nbytes // dt.itemsize if count is None else int(count)
        if n * dt.itemsize > self.nbytes:
            raise ValueError("view larger than the buffer")
        raw = (ctypes.c_char * (n * dt.itemsize)).from_address(self.ptr)
        return np.frombuffer(raw, dtype=dt, count=n)

    def close(self):
        if self.ptr:
            prng_host_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prng_destroy(h):
    lib().prng_destroy(h)


class Generator:
    """A handle of n_streams streams of one generator, owned by this object."""

    def __init__(self, gen, seed: int, n_streams: int, luxury: int = 0):
        self.gen = _gen(gen)
        self.n_streams = n_streams
        self.luxury = luxury
        self._h = prng_create(self.gen, seed, n_streams, luxury)

    @property
    def handle(self):
        return self._h

    def fill(self, n_per_stream: int, dtype: str = "u32", out=None, stream=None):
        """Next n_per_stream outputs of every stream as a (n_streams,
        n_per_stream) CUDA tensor: int32 holding the u32 bits, float32, or
        float64 (each double made of two draws)."""
        import torch
        if out is None:
            tdt = {"f32": torch.float32, "f64": torch.float64}.get(dtype, torch.int32)
            out = torch.empty((self.n_streams, n_per_stream), dtype=tdt, device="cuda")
        if dtype == "f32":
            prng_fill_f32(self._h, out, n_per_stream, stream)
        elif dtype == "f64":
            prng_fill_f64(self._h, out, n_per_stream, stream)
        else:
            prng_fill_u32(self._h, out, n_per_stream, stream)
        return out

    def skip(self, k: int, stream=None):
        prng_skip(self._h, k, stream)

    def reseed(self, seed: int, stream=None):
        prng_reseed(self._h, seed, stream)

    def get_state(self) -> bytes:
        return prng_get_state(self._h)

    def set_state(self, blob: bytes):
        prng_set_state(self._h, blob)

    def close(self):
        if self._h is not None and self._h.value:
            prng_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
