"""Benchmark of the bulk-generation hot path on GB300.

One step = one pass of the whole path over the roofline workload:
  * re-seed every stream of the six handles on the device;
  * GGL, XOR128, RANECU, RANMAR, RANLUX (p = 24) fill 2^30 u32 and 2^30 f32
    each over 131,072 streams (8,192 per stream); MT19937 the same over
    8,192 streams (131,072 per stream);
  * GGL and RANECU jump-ahead fill 2^30 draws of one sequence from x0 = 1
    in 65,536 chunks.
value = random numbers written per second (whole job, all ranks).  Outputs
(4 GiB per buffer) are far larger than L2, so no flush is needed between
steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the paper's plain single-threaded
definitions) on this machine's host cores on a bounded sample of the same
workload mix.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GENS = ("ggl", "xor128", "ranecu", "ranmar", "ranlux", "mt19937")
N_STREAMS = 131072
N_PER = 8192
MT_STREAMS = 8192
MT_PER = 131072
JUMP_N = 2**30
JUMP_CHUNKS = 65536
JUMP_X0 = {"ggl": 1, "ranecu": 1 | (1 << 32)}
SEED = 0x5EED
RANLUX_P = 24
STATE_WORDS = {"ggl": 1, "xor128": 4, "ranecu": 2, "ranmar": 98, "ranlux": 25, "mt19937": 624}
METRIC = "random numbers/s per generator (and % of HBM-write roofline); batched p50/p99 latency"
WORKLOAD = ("roofline bulk fill: GGL, XOR128, RANECU, RANMAR, RANLUX p=24 each 2^30 u32 + 2^30 f32 "
            "over 131072 streams; MT19937 2^30 u32 + 2^30 f32 over 8192 streams; GGL and RANECU "
            "jump-ahead 2^30 draws from x0=1 in 65536 chunks; streams re-seeded each step")


def shape(gen):
    return (MT_STREAMS, MT_PER) if gen == "mt19937" else (N_STREAMS, N_PER)


def step_items():
    """(label, generator, kind, numbers) for one step, in launch order."""
    items = []
    for g in GENS:
        ns, nper = shape(g)
        items.append((f"{g}_u32", g, "u32", ns * nper))
        items.append((f"{g}_f32", g, "f32", ns * nper))
    for g in ("ggl", "ranecu"):
        items.append((f"{g}_jump", g, "jump", JUMP_N))
    return items


def numbers_per_step():
    return sum(n for _, _, _, n in step_items())


def algorithmic_bytes(label, gen, kind, numbers):
    """Bytes a launch must move: 4 B per output plus one read and one write
    of the stream state (a jump chunk's state is computed, not loaded)."""
    if kind == "jump":
        return 4 * numbers
    ns, _ = shape(gen)
    return 4 * numbers + 2 * 4 * STATE_WORDS[gen] * ns


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Device sources that make up each generator's fill kernels (besides the
# shared headers).  Which of them a launch runs is set by the launch tile,
# which the recorded traffic is keyed on as well.
KERNEL_SOURCES = {
    "ggl": ["k_mlcg.cu", "k_simple.cu"], "ranecu": ["k_mlcg.cu", "k_simple.cu"],
    "xor128": ["k_simple.cu"], "ranmar": ["k_ranmar.cu"],
    "ranlux": ["ranlux.cuh", "k_ranlux.cu", f"k_ranlux_p{RANLUX_P}.cu"], "mt19937": ["k_mt.cu"],
}
SHARED_SOURCES = ["common.cuh", "batch.cuh"]


def _code_only(text: str) -> str:
    """C/C++ source without its comments and with whitespace collapsed, so
    that the hash below follows the code, not its comments."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sources_hash(gen):
    """Hash of the code (comments and layout ignored) of the sources a
    generator's fill kernels are built from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1003_1898_gb300", "csrc")
    for fn in SHARED_SOURCES + KERNEL_SOURCES[gen]:
        with open(os.path.join(csrc, fn), encoding="utf-8") as f:
            h.update(fn.encode() + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(label, gen, tile=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current sources of that generator's kernels and (when given) with
    the launch tile in effect now; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
        entry = t["per_launch"].get(label)
        if entry is None or entry.get("sources") != kernel_sources_hash(gen):
            return None
        if tile is not None and list(entry.get("tile", [])) != list(tile):
            return None
        return entry["bytes"]
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


class NvmlClockSampler:
    """The same record read through NVML (read-only queries: current and
    maximum SM clock, active clock-event reasons) every 5 ms, so that a
    timed region of a few tens of milliseconds still gets several samples.
    The device is found by its UUID."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid: str):
        import ctypes
        self.ct = ctypes
        self.nv = ctypes.CDLL("libnvidia-ml.so.1")
        if self.nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.nv.nvmlDeviceGetHandleByUUID(("GPU-" + uuid).encode(), ctypes.byref(self.h)) != 0:
            raise RuntimeError("NVML has no device with this UUID")
        try:
            self.get_reasons = self.nv.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self.get_reasons = self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 \
            else None
        self.samples = []
        self.stop = threading.Event()

    def _loop(self):
        ct = self.ct
        mhz, rs = ct.c_uint(), ct.c_ulonglong()
        while not self.stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz)) == 0 and \
                    self.get_reasons(self.h, ct.byref(rs)) == 0:
                self.samples.append((float(mhz.value), int(rs.value)))
            time.sleep(0.005)

    def __enter__(self):
        self.t = threading.Thread(target=self._loop, daemon=True)
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.t.join(timeout=5)
        self.nv.nvmlShutdown()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0,
                    "source": "nvml"}
        reasons = sorted({name for _, r in self.samples for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(m for m, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(self.samples), "source": "nvml"}


def clock_sampler(torch, dev, local_rank):
    """NVML sampling when the driver's library is there, else nvidia-smi."""
    try:
        return NvmlClockSampler(str(torch.cuda.get_device_properties(dev).uuid))
    except Exception:
        return ClockSampler(local_rank)


# ------------------------------------------------------------------ oracle arm

def cpu_oracle_rate(sample_per_item: int):
    """Oracle (single thread) numbers/s on the step's mix: each item draws
    `sample_per_item` numbers; the mix rate is total numbers / total time,
    with every item weighted by its share of the step."""
    import oracle
    oracle.lib()
    t_total = 0.0
    n_total = 0
    for label, g, kind, numbers in step_items():
        t0 = time.perf_counter()
        if kind == "jump":
            oracle.serial_fill(g, JUMP_X0[g], sample_per_item)
        else:
            lux = RANLUX_P if g == "ranlux" else 0
            # u32 and f32 share the integer draws; f32 adds one exact conversion
            if kind == "f32":
                u, f = oracle.fill(g, SEED, 1, sample_per_item, luxury=lux, want_f32=True)
            else:
                oracle.checksum_draws(g, SEED, 0, sample_per_item, luxury=lux)
        dt = time.perf_counter() - t0
        t_total += dt * (numbers / sample_per_item)
        n_total += numbers
    return n_total / t_total, t_total


def cpu_oracle_rate_threads(sample_per_item: int, threads: int):
    """The same mix with every item split over `threads` host threads (the
    oracle's C functions release the GIL): thread t draws its share from its
    own stream (jump items: its own serial sequence).  Returns numbers/s."""
    import concurrent.futures as cf
    import oracle
    oracle.lib()
    per = max(1, sample_per_item // threads)
    t_total = 0.0
    n_total = 0
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for label, g, kind, numbers in step_items():
            lux = RANLUX_P if g == "ranlux" else 0
            if kind == "jump":
                work = lambda t: oracle.serial_fill(g, JUMP_X0[g] + 2 * t, per)
            elif kind == "f32":
                work = lambda t: oracle.fill(g, SEED, 1, per, luxury=lux, stream0=t, want_f32=True)
            else:
                work = lambda t: oracle.checksum_draws(g, SEED, t, per, luxury=lux)
            t0 = time.perf_counter()
            list(ex.map(work, range(threads)))
            dt = time.perf_counter() - t0
            t_total += dt * (numbers / (per * threads))
            n_total += numbers
    return n_total / t_total


def rank_seed_base(g: str, rank: int) -> int:
    """Rank `rank` owns streams [rank n, (rank + 1) n) of one handle of
    world * n streams (n = this generator's stream count): stream i of a
    handle is seeded from base + i, so its base is SEED + rank * n."""
    return SEED + rank * shape(g)[0]


def rank_jump_first(rank: int) -> int:
    """Rank `rank`'s jump fills cover draws [rank N, (rank + 1) N) of the one
    sequence from x0 (N = JUMP_N), so that the ranks tile it."""
    return rank * JUMP_N


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time (all-reduce MAX; a CUDA tensor under NCCL)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    """The oracle as the reference arm.  Every item of the GPU step has the
    same count (2^30 numbers), so a step here is the same mix scaled down:
    each item draws `cpu_sample` numbers.  ms_per_step is that sampled
    step's own wall time, and value is the numbers it drew over that time."""
    if rank != 0:
        return
    sample = args.cpu_sample
    items = step_items()
    assert len({n for *_, n in items}) == 1, "the sample assumes equal item counts"
    per_step = sample * len(items)
    steps_t = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cpu_oracle_rate(sample)
        if i >= args.warmup:
            steps_t.append(time.perf_counter() - t0)
    secs = statistics.median(steps_t)
    rate = per_step / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "numbers/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "sample": f"each step is the workload's mix scaled down: {sample} numbers per "
                             f"step item ({len(items)} items, {per_step} numbers per step); "
                             "ms_per_step is that step's own time",
                   "numbers_per_step": per_step},
        "cpu_baseline": {"value": rate, "unit": "numbers/s", "cores": 1, "kind": "oracle",
                         "sample": f"{sample} draws per step item, single thread"},
        "e2e": {"value": rate, "unit": "numbers/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

LUX_STREAMS, LUX_PER = 65536, 4096
SWB_CHAIN_OPS = 24 * 2 + 3  # one 24-step chain: 24 subtract-with-borrow, 24 clears, 3 flag moves


def _time_ms(torch, stream, fn, reps=5, warm=2):
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def measure_xor128_jump(P, torch, out_u, h_xor, stream):
    """XOR128 jump-ahead over GF(2): the single-sequence fill of 2^30 draws
    in 65,536 chunks (chunk starts by doubling passes of T^L, then the
    ordinary fill), and prng_skip(2^40) of the 131,072-stream handle."""
    sid = stream.cuda_stream
    x0 = SEED
    ms = _time_ms(torch, stream, lambda: P.prng_fill_jump_u32("xor128", x0, JUMP_N, JUMP_CHUNKS,
                                                               out_u.data_ptr(), sid))
    byt = 4 * JUMP_N
    skip_ms = _time_ms(torch, stream, lambda: P.prng_skip(h_xor, 2**40, sid))
    return {"fill": {"numbers": JUMP_N, "chunks": JUMP_CHUNKS, "ms": ms,
                     "numbers_per_s": JUMP_N / (ms / 1e3), "gbs": byt / (ms / 1e3) / 1e9,
                     "frac_hbm": byt / (ms / 1e3) / 1e9 / peaks()[0]},
            "skip_2p40": {"streams": N_STREAMS, "ms": skip_ms}}


def measure_ising_fused(P, torch, out_u, stream, L=4096):
    """Checkerboard Metropolis sweeps of a 4096 x 4096 lattice: the draws
    stored (prng_fill_u32 then prng_ising_half_sweep, the serving path) or
    consumed where they are made (prng_ising_fused), per generator and
    stream count.  ms per sweep (two half-sweeps, 2^24 site updates)."""
    sid = stream.cuda_stream
    t4, t8 = P.prng_ising_thresholds(0.4406868)
    spins = torch.ones((L, L), dtype=torch.int8, device=out_u.device)
    draws = out_u[: L * L // 2]
    res = {"L": L, "runs": []}
    for g, lux, ns in [("ggl", 0, 1024), ("ggl", 0, 65536), ("xor128", 0, 65536),
                       ("ranecu", 0, 65536), ("ranmar", 0, 65536), ("ranlux", 223, 65536),
                       ("mt19937", 0, 8192)]:
        h = P.prng_create(g, SEED, ns, lux)
        per = L * L // (2 * ns)

        def stored():
            for colour in (0, 1):
                P.prng_fill_u32(h, draws.data_ptr(), per, sid)
                P.prng_ising_half_sweep([{"d_spins": spins, "d_draws": draws, "L": L,
                                          "colour": colour, "gen": g, "t4": t4, "t8": t8}], sid)

        def fused():
            for colour in (0, 1):
                P.prng_ising_fused(h, spins, L, colour, t4, t8, sid)

        ms_s = _time_ms(torch, stream, stored, reps=5, warm=2)
        ms_f = _time_ms(torch, stream, fused, reps=5, warm=2)
        P.prng_destroy(h)
        res["runs"].append({"gen": g, "luxury": lux, "streams": ns, "ms_per_sweep_stored": ms_s,
                            "ms_per_sweep_fused": ms_f,
                            "site_updates_per_s_fused": L * L / (ms_f / 1e3)})
    return res


def measure_mt_jump(P, torch, out_u, h_mt, stream):
    """MT19937 jump-ahead over GF(2): prng_skip(2^40) of the 8,192-stream
    handle (the jump polynomial applied to every table), and the
    single-sequence fill of 2^30 draws from init_genrand(5489) in 8,192
    chunks (chunk starts by doubling passes, then the ordinary fill)."""
    sid = stream.cuda_stream
    skip_ms = _time_ms(torch, stream, lambda: P.prng_skip(h_mt, 2**40, sid), reps=3, warm=1)
    ms = _time_ms(torch, stream, lambda: P.prng_fill_jump_u32("mt19937", 5489, JUMP_N, MT_STREAMS,
                                                               out_u.data_ptr(), sid), reps=3, warm=1)
    return {"skip_2p40": {"streams": MT_STREAMS, "ms": skip_ms},
            "fill": {"numbers": JUMP_N, "chunks": MT_STREAMS, "ms": ms,
                     "numbers_per_s": JUMP_N / (ms / 1e3),
                     "frac_hbm": 4 * JUMP_N / (ms / 1e3) / 1e9 / peaks()[0]}}


def measure_f64(P, torch, out_u, handles, seed_r, stream):
    """Doubles from pairs of draws: 2^29 doubles (4 GiB) per generator on
    the roofline handles, each double made of two draws; bytes per launch
    are the 8-byte outputs plus the state read and write."""
    sid = stream.cuda_stream
    res = {}
    for g in GENS:
        ns, nper = shape(g)
        P.prng_reseed(handles[g], seed_r[g], sid)
        ms = _time_ms(torch, stream, lambda: P.prng_fill_f64(handles[g], out_u.data_ptr(), nper // 2, sid))
        n = ns * (nper // 2)
        byt = 8 * n + 2 * 4 * STATE_WORDS[g] * ns
        res[g] = {"doubles": n, "ms": ms, "doubles_per_s": n / (ms / 1e3),
                  "gbs": byt / (ms / 1e3) / 1e9, "frac_hbm": byt / (ms / 1e3) / 1e9 / peaks()[0]}
    return res


def measure_swb_rate(P, torch, dev, stream):
    """The integer rate of the RANLUX kernels' own subtract-with-borrow chain,
    measured (prng_calib_swb): throughput with four independent chains per
    thread at full occupancy, and latency with one chain per thread and one
    warp per scheduler (4 per SM).  Clocks are sampled during the timed
    launches, so the rate is also given per SM per clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(sms * 2048, dtype=torch.int32, device=dev)
    sid = stream.cuda_stream
    res = {"sm_count": sms, "chain_instructions": SWB_CHAIN_OPS}
    with clock_sampler(torch, dev, dev.index or 0) as clk:
        for name, chains, warps, iters in (("throughput", 4, 0, 8192), ("throughput_2", 2, 0, 8192),
                                           ("latency", 1, 4, 4096)):
            ops = [0]

            def run():
                ops[0] = P.prng_calib_swb(chains, warps, iters, sink, sid)
            ms = _time_ms(torch, stream, run, reps=5, warm=2)
            res[name] = {"chains_per_thread": chains, "warps_per_sm": warps or "max",
                         "iters": iters, "ms": ms, "ops": ops[0], "ops_per_s": ops[0] / (ms / 1e3)}
    c = clk.summary()
    mhz = c.get("sm_mhz") or 2070.0
    res["clocks"] = c
    for name in ("throughput", "throughput_2", "latency"):
        r = res[name]
        r["ops_per_sm_clk"] = r["ops_per_s"] / (sms * mhz * 1e6)
    # one warp per scheduler, one chain per thread: cycles per SWB step
    lat = res["latency"]
    lat["cycles_per_step"] = (lat["ms"] / 1e3) * mhz * 1e6 / (lat["iters"] * 24)
    res["bound_ops_per_s"] = max(res["throughput"]["ops_per_s"], res["throughput_2"]["ops_per_s"])
    return res


def measure_luxury_sweep(P, torch, dev, stream, sm_mhz):
    """ns/number of RANLUX f32 fills (2^28 over 65,536 streams) for every
    standard p, and the fraction of the integer-pipe bound reached.  The
    bound counts the subtract-with-borrow chains alone: p/24 steps per
    delivered number, each one subtract-with-borrow plus one low-byte clear,
    plus 3 instructions per 24-step chain to move the borrow in and out of
    the carry flag, at the rate that same chain is measured to run at on
    this GPU with its latency hidden (measure_swb_rate)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_mhz or 2070.0
    swb = measure_swb_rate(P, torch, dev, stream)
    rate = swb["bound_ops_per_s"]
    out = torch.empty(LUX_STREAMS * LUX_PER, dtype=torch.float32, device=dev)
    res = {"workload": f"{LUX_STREAMS} streams x {LUX_PER} f32 per p (2^28 numbers)",
           "sm_count": sms, "sm_mhz": mhz, "swb_chain_rate": swb,
           "bound_source": "measured: prng_calib_swb throughput (same chain, latency hidden)",
           "levels": {}}
    for p in (24, 48, 97, 223, 389, 120, 240, 408):
        h = P.prng_create("ranlux", SEED, LUX_STREAMS, p)
        sid = stream.cuda_stream
        for _ in range(2):
            P.prng_fill_f32(h, out.data_ptr(), LUX_PER, sid)
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            P.prng_fill_f32(h, out.data_ptr(), LUX_PER, sid)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        P.prng_destroy(h)
        ms = statistics.median(ts)
        n = LUX_STREAMS * LUX_PER
        instr = (p / 24.0) * SWB_CHAIN_OPS / 24.0
        bound_ms = 1e3 * n * instr / rate
        hbm_ms = 1e3 * 4 * n / (peaks()[0] * 1e9)
        res["levels"][str(p)] = {"ms": ms, "ns_per_number": 1e6 * ms / n, "numbers_per_s": n / (ms / 1e3),
                                 "int_instr_per_number": instr, "int_bound_ms": bound_ms,
                                 "hbm_bound_ms": hbm_ms,
                                 "frac_of_bound": max(bound_ms, hbm_ms) / ms,
                                 "bound": "alu" if bound_ms > hbm_ms else "hbm"}
    del out
    return res


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_1003_1898_gb300 as P
    from paper_1003_1898_gb300 import build as B

    torch.cuda.set_device(local_rank)
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    P.lib()
    from paper_1003_1898_gb300 import tune as TU
    tuned = TU.load_and_apply()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream

    # Each rank owns disjoint streams: seed bases offset by the stream count.
    seed_r = {g: rank_seed_base(g, rank) for g in GENS}
    handles = {g: P.prng_create(g, seed_r[g], shape(g)[0], RANLUX_P if g == "ranlux" else 0)
               for g in GENS}
    out_u = torch.empty(N_STREAMS * N_PER, dtype=torch.int32, device=dev)
    out_f = torch.empty(N_STREAMS * N_PER, dtype=torch.float32, device=dev)
    items = step_items()
    ev = {lab: [] for lab, *_ in items}

    def one_step(record):
        for g in GENS:
            P.prng_reseed(handles[g], seed_r[g], sid)
        for lab, g, kind, numbers in items:
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            if kind == "u32":
                P.prng_fill_u32(handles[g], out_u.data_ptr(), shape(g)[1], sid)
            elif kind == "f32":
                P.prng_fill_f32(handles[g], out_f.data_ptr(), shape(g)[1], sid)
            else:
                P.prng_fill_jump_at_u32(g, JUMP_X0[g], rank_jump_first(rank), JUMP_N, JUMP_CHUNKS,
                                        out_u.data_ptr(), sid)
            if record:
                e1.record(stream)
                ev[lab].append((e0, e1))

    for _ in range(args.warmup):
        one_step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with clock_sampler(torch, dev, local_rank) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            one_step(True)
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms_total = t0.elapsed_time(t1)
    if world > 1:
        ms_total = max_over_ranks(ms_total, dist, dev)
    ms_step = ms_total / args.steps
    value = world * numbers_per_step() / (ms_step / 1e3)
    launches_per_step = len(GENS) + len(items)

    # per-item device time (events on the launching stream) and roofline
    hbm, peak_kind = peaks()
    per = {}
    for lab, g, kind, numbers in items:
        ts = [a.elapsed_time(b) for a, b in ev[lab]]
        ms = statistics.mean(ts)
        byt = algorithmic_bytes(lab, g, kind, numbers)
        per[lab] = {"ms": ms, "numbers_per_s": numbers / (ms / 1e3),
                    "gbs": byt / (ms / 1e3) / 1e9, "frac_hbm": byt / (ms / 1e3) / 1e9 / hbm}
    dom = max(items, key=lambda it: per[it[0]]["ms"])
    dl = dom[0]
    roof = {"kernel": dl, "bound": "hbm", "achieved": per[dl]["gbs"], "peak": hbm,
            "unit": "GB/s", "frac": per[dl]["frac_hbm"],
            "traffic": recorded_traffic(dl, dom[1], P.prng_get_tile(dom[1], RANLUX_P if dom[1] == "ranlux" else 0)),
            "peak_source": f"{peak_kind} hbm_gbs (copy, read+write)",
            "algorithmic_bytes_per_launch": algorithmic_bytes(*dom)}

    # Write-only ceiling for context: torch's own fill kernel over the same
    # 4 GiB buffer (a plain store stream with no generator arithmetic; a
    # non-zero value, so it is a kernel and not a memset).
    wo = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out_u.fill_(0x1234567)
        b.record(stream)
        torch.cuda.synchronize()
        wo.append(a.elapsed_time(b))
    write_only_gbs = 4 * out_u.numel() / (statistics.median(wo) / 1e3) / 1e9
    roof["write_only_gbs"] = write_only_gbs
    roof["frac_of_write_only"] = per[dl]["gbs"] / write_only_gbs

    # RANLUX luxury sweep: 2^28 f32 per p over 65,536 streams, against the
    # integer-pipe bound of the subtract-with-borrow chains.
    lux_sweep = measure_luxury_sweep(P, torch, dev, stream, clk.summary().get("sm_mhz"))
    xor128_jump = measure_xor128_jump(P, torch, out_u, handles["xor128"], stream)
    f64 = measure_f64(P, torch, out_u, handles, seed_r, stream)
    mt_jump = measure_mt_jump(P, torch, out_u, handles["mt19937"], stream)
    ising_fused = measure_ising_fused(P, torch, out_u, stream)

    # Batched requests (20,000 mixed fills): one graph launch vs one plain
    # re-seed + fill per request.
    batched = None
    if not args.no_batched:
        del out_u, out_f
        out_u = out_f = None
        torch.cuda.empty_cache()
        batched = measure_batched(P, dev, args)

    # Serving loop (512 clients, Poisson arrivals, fills and Ising runs):
    # continuous batching vs a plain one-request-at-a-time queue.
    serving = None
    if not args.no_serving:
        serving = measure_serving(args)

    # end-to-end through the public API with host buffers: fill, then copy
    # every output to pinned host memory inside the timed region.
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(P, handles, seed_r, items, dev, args, rank)

    for h in handles.values():
        P.prng_destroy(h)
    if rank != 0:
        return
    cpu = cpu_mt = None
    if world == 1 and not args.no_cpu:
        rate, secs = cpu_oracle_rate(args.cpu_sample)
        cpu = {"value": rate, "unit": "numbers/s", "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_sample} draws per step item ({len(items)} items), single "
                         f"thread, weighted by the step's mix"}
        nthr = os.cpu_count() or 1
        rate_mt = cpu_oracle_rate_threads(args.cpu_sample, nthr)
        cpu_mt = {"value": rate_mt, "unit": "numbers/s", "cores": nthr, "kind": "oracle",
                  "sample": f"{args.cpu_sample} draws per step item split over {nthr} threads "
                            f"(one stream each), weighted by the step's mix"}
    line = {
        "metric": METRIC, "value": value, "unit": "numbers/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "numbers_per_step_per_gpu": numbers_per_step(),
                   "l2": "outputs (4 GiB per buffer) larger than L2; no flush",
                   "parallelism": f"{world} independent partitions of the streams"},
        "clocks": clk.summary(),
        "e2e": e2e,
        "batched": batched,
        "serving": serving,
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_mt,
        "per_kernel": per,
        "luxury_sweep": lux_sweep,
        "xor128_jump": xor128_jump,
        "f64": f64,
        "mt_jump": mt_jump,
        "ising_fused": ising_fused,
        "tiles": {"tuned_cache": bool(tuned),
                  **{g: list(P.prng_get_tile(g, RANLUX_P if g == "ranlux" else 0)) for g in GENS}},
    }
    print(json.dumps(line), flush=True)


def measure_batched(P, dev, args):
    """Config of 20,000 requests: lengths log-uniform in [1e2, 1e7], generator
    uniform over the six (RANLUX p = 223), u32/f32 at random.  Both forms
    re-seed every request's streams and fill them; the outputs are the same
    bytes.  Latency of a request = its completion time after the first
    launch of the pass (per-request events for the plain form; every request
    of a batch completes with the batch)."""
    import torch
    from paper_1003_1898_gb300 import workloads as W
    reqs = W.batched_requests(args.batch_requests)
    sizes = [((q["n_streams"] * q["n_per"] + 3) // 4) * 4 for q in reqs]
    offs = [0]
    for z in sizes:
        offs.append(offs[-1] + z)
    buf = torch.empty(offs[-1], dtype=torch.int32, device=dev)
    base = buf.data_ptr()
    handles = [P.prng_create(q["gen"], q["seed"], q["n_streams"], q["luxury"]) for q in reqs]
    fr = [{"st": h, "d_out": base + 4 * o, "n_per_stream": q["n_per"], "n_valid": q["n"],
           "f32": q["f32"], "reseed": True, "seed": q["seed"]}
          for h, q, o in zip(handles, reqs, offs)]
    b = P.prng_batch_create(fr)
    info = P.prng_batch_info(b)
    numbers = info["numbers"]
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # batched: one graph launch per pass
    for _ in range(2):
        P.prng_batch_launch(b, sid)
    torch.cuda.synchronize()
    bt = []
    for _ in range(args.batch_passes):
        e0, e1 = ev(), ev()
        e0.record(stream)
        P.prng_batch_launch(b, sid)
        e1.record(stream)
        torch.cuda.synchronize()
        bt.append(e0.elapsed_time(e1))
    # plain: re-seed and fill each request with its own launches
    def plain(record):
        done = []
        e0 = ev()
        e0.record(stream)
        for h, q, o in zip(handles, reqs, offs):
            P.prng_reseed(h, q["seed"], sid)
            (P.prng_fill_f32 if q["f32"] else P.prng_fill_u32)(h, base + 4 * o, q["n_per"], sid)
            if record:
                e = ev()
                e.record(stream)
                done.append(e)
        e1 = ev()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0, e1, done
    plain(False)
    pt, lat = [], []
    for i in range(args.batch_passes):
        t_host = time.perf_counter()
        e0, e1, done = plain(i == 0)
        pt.append(max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t_host)))
        if done:
            lat = sorted(e0.elapsed_time(e) for e in done)
    # The same two forms without the re-seed: fills only (every pass
    # continues the streams, so the bytes differ between passes; the work
    # does not).
    fr_ns = [dict(r, reseed=False) for r in fr]
    b_ns = P.prng_batch_create(fr_ns)
    for _ in range(2):
        P.prng_batch_launch(b_ns, sid)
    torch.cuda.synchronize()
    bt_ns = []
    for _ in range(args.batch_passes):
        e0, e1 = ev(), ev()
        e0.record(stream)
        P.prng_batch_launch(b_ns, sid)
        e1.record(stream)
        torch.cuda.synchronize()
        bt_ns.append(e0.elapsed_time(e1))
    P.prng_batch_destroy(b_ns)
    pt_ns = []
    for _ in range(args.batch_passes):
        t_host = time.perf_counter()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for h, q, o in zip(handles, reqs, offs):
            (P.prng_fill_f32 if q["f32"] else P.prng_fill_u32)(h, base + 4 * o, q["n_per"], sid)
        e1.record(stream)
        torch.cuda.synchronize()
        pt_ns.append(max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t_host)))
    P.prng_batch_destroy(b)
    for h in handles:
        P.prng_destroy(h)
    del buf
    torch.cuda.empty_cache()
    bms, pms = statistics.median(bt), statistics.median(pt)
    bns, pns = statistics.median(bt_ns), statistics.median(pt_ns)
    pct = lambda xs, q: xs[min(len(xs) - 1, int(q * len(xs)))]
    return {"requests": len(reqs), "numbers_per_pass": numbers, "work_items": info["items"],
            "batched": {"ms_per_pass": bms, "numbers_per_s": numbers / (bms / 1e3),
                        "p50_ms": bms, "p99_ms": bms, "launches_per_pass": 1},
            "per_request": {"ms_per_pass": pms, "numbers_per_s": numbers / (pms / 1e3),
                            "p50_ms": pct(lat, 0.50) if lat else None,
                            "p99_ms": pct(lat, 0.99) if lat else None,
                            "launches_per_pass": 2 * len(reqs)},
            "speedup": pms / bms,
            "without_seeding": {
                "batched": {"ms_per_pass": bns, "numbers_per_s": numbers / (bns / 1e3),
                            "launches_per_pass": 1},
                "per_request": {"ms_per_pass": pns, "numbers_per_s": numbers / (pns / 1e3),
                                "launches_per_pass": len(reqs)},
                "speedup": pns / bns},
            "note": "per-request time is the larger of the device span and the host "
                    "enqueue time of its launches; the main figures re-seed every request "
                    "inside the pass, without_seeding times the fills alone"}


def measure_serving(args):
    """512 clients with device-resident streams (half RANLUX p = 223), Poisson
    arrivals at each rate, requests 50/50 a fill of 1e3..1e6 numbers or 16
    checkerboard sweeps of an L x L Ising lattice (L in {256, 1024, 4096}),
    40 GB state + output cap.  Aggregate numbers/s counts every draw served
    (fill outputs and Ising draws).  At every rate the same arrivals are
    served twice: with continuous batching, and by a plain queue that runs
    one request at a time (the one-launch-per-request baseline)."""
    from paper_1003_1898_gb300 import serve as S
    from paper_1003_1898_gb300 import workloads as W
    specs = W.serving_clients(W.SERVE_CLIENTS)
    streams = getattr(args, "serve_streams", None) or W.SERVE_STREAMS
    out = {"clients": W.SERVE_CLIENTS, "streams_per_client": streams,
           "mem_cap_bytes": W.SERVE_MEM_CAP, "half_sweeps_per_tick": args.serve_hpt,
           "rates": []}
    arms = [a for a in ("continuous", "queue") if a in args.serve_arms]
    for rate in args.serve_rates:
        row = {"rate_per_s": rate, "requests": args.serve_requests}
        raw = W.serving_requests(args.serve_requests, rate)
        for mode in arms:
            srv = S.Server(specs, n_streams=streams, mem_cap=W.SERVE_MEM_CAP,
                           max_active=1 if mode == "queue" else 0,
                           half_sweeps_per_tick=args.serve_hpt)
            try:
                srv.run([S.Request(**r) for r in raw[: min(50, len(raw))]],
                        realtime=False)   # warm-up (compile, caches)
                done = srv.run([S.Request(**r) for r in raw], realtime=True)
            finally:
                srv.close()
            row[mode] = S.latency_stats(done)
            # where a tick's time goes: host work per tick, and the GPU time of
            # its fills and half-sweeps, against the run's span
            row[mode]["ticks"] = srv.stats["ticks"]
            row[mode]["host_launch_s"] = srv.stats["launch_s"]
            row[mode]["host_batcher_s"] = srv.stats["batcher_s"]
            row[mode]["gpu_tick_s"] = srv.stats["gpu_s"]
        out["rates"].append(row)
    return out


def serving_main(argv):
    """The serving sweep alone: bench.py serving [--rates R ...] [--requests N]
    [--arms continuous queue] [--hpt H] [--streams S].  Prints one JSON line."""
    import torch
    import paper_1003_1898_gb300 as P
    from paper_1003_1898_gb300 import build as B
    from paper_1003_1898_gb300 import tune
    ap = argparse.ArgumentParser(prog="bench.py serving")
    ap.add_argument("--rates", dest="serve_rates", type=float, nargs="+",
                    default=[500.0, 1000.0, 1500.0, 2000.0, 2500.0, 3000.0, 4000.0, 8000.0, 16000.0])
    ap.add_argument("--requests", dest="serve_requests", type=int, default=10000)
    ap.add_argument("--arms", dest="serve_arms", nargs="+", default=["continuous", "queue"])
    ap.add_argument("--hpt", dest="serve_hpt", type=int, default=4)
    ap.add_argument("--streams", dest="serve_streams", type=int, default=None,
                    help="streams per client (default: the workload's)")
    a = ap.parse_args(argv)
    B.build()
    P.lib()
    tune.load_and_apply()
    dev = torch.device("cuda", 0)
    with clock_sampler(torch, dev, 0) as clk:
        res = measure_serving(a)
    res["clocks"] = clk.summary()
    print(json.dumps(res), flush=True)


def measure_e2e(P, handles, seed_r, items, dev, args, rank=0):
    """The step end to end through the C ABI with host outputs: every fill
    writes its numbers into page-locked host memory from prng_host_alloc, so
    the kernels' stores cross the host link (NVLink-C2C) and no device
    staging buffer or copy is involved.  Wall-clock over whole steps,
    synchronised at both ends.  For context, one 4 GiB copy-engine transfer
    (device buffer to pinned host tensor) is timed too."""
    import torch
    stream = torch.cuda.current_stream()
    host = P.HostBuffer(4 * N_STREAMS * N_PER)
    d2h = 0
    steps = max(1, args.steps)            # the same K steps as the device-timed figure

    def one():
        nonlocal d2h
        for g in GENS:
            P.prng_reseed(handles[g], seed_r[g], stream.cuda_stream)
        for lab, g, kind, numbers in items:
            if kind == "u32":
                P.prng_fill_u32(handles[g], host.ptr, shape(g)[1], stream.cuda_stream)
            elif kind == "f32":
                P.prng_fill_f32(handles[g], host.ptr, shape(g)[1], stream.cuda_stream)
            else:
                P.prng_fill_jump_at_u32(g, JUMP_X0[g], rank_jump_first(rank), JUMP_N, JUMP_CHUNKS,
                                        host.ptr, stream.cuda_stream)
            d2h += 4 * numbers

    try:
        one()
        torch.cuda.synchronize()
        d2h = 0
        t0 = time.perf_counter()
        for _ in range(steps):
            one()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / steps
        d2h //= steps
        src = torch.empty(N_STREAMS * N_PER, dtype=torch.int32, device=dev)
        pinned = torch.empty(N_STREAMS * N_PER, dtype=torch.int32, pin_memory=True)
        pinned.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        ce_ms = _time_ms(torch, stream, lambda: pinned.copy_(src, non_blocking=True), reps=3, warm=1)
        del src, pinned
    finally:
        host.close()
    return {"value": numbers_per_step() / dt, "unit": "numbers/s",
            "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
            "host_link_gbs": d2h / dt / 1e9,
            "copy_engine_gbs": 4 * N_STREAMS * N_PER / ce_ms / 1e6,
            "note": "fills through the C ABI writing straight into page-locked host memory "
                    "(prng_host_alloc); inputs are scalar seeds passed by value; "
                    "copy_engine_gbs is one 4 GiB device-to-pinned-host copy for context"}


# ------------------------------------------------------------ single kernels

def kernel_main(argv):
    """One kernel in isolation (CUDA events), for tile studies and profiler
    captures of a single launch:

      bench.py kernel fill GEN {u32,f32,f64} N_STREAMS N_PER [--luxury P]
          [--reps R] [--timed K] [--jump] [--skip] [--tile T,C,S]
      bench.py kernel ising L N_LATTICES [--reps R] [--timed K]
      bench.py kernel fused GEN L N_STREAMS [--luxury P] [--reps R] [--timed K]

    fill: one fill of GEN (--jump: the single-sequence jump fill, N_STREAMS
    chunks of N_PER draws; --skip: prng_skip of N_PER draws per stream; f64:
    N_PER doubles per stream).  The tuned tiles are applied first, then
    --tile for GEN.  ising: one batched half-sweep launch over N_LATTICES
    cold-start lattices of side L with random draws (colour 0).  fused: one
    fused half-sweep (prng_ising_fused) of a cold-start L x L lattice on a
    handle of N_STREAMS streams.  Prints one line per timed call."""
    import numpy as np
    import torch

    import paper_1003_1898_gb300 as P
    from paper_1003_1898_gb300 import build as B
    from paper_1003_1898_gb300 import tune
    from paper_1003_1898_gb300.workloads import JUMP_X0 as JX0
    ap = argparse.ArgumentParser(prog="bench.py kernel")
    sub = ap.add_subparsers(dest="what", required=True)
    f = sub.add_parser("fill")
    f.add_argument("gen", choices=sorted(P.GEN_IDS))
    f.add_argument("dtype", choices=["u32", "f32", "f64"])
    f.add_argument("n_streams", type=int)
    f.add_argument("n_per", type=int)
    f.add_argument("--jump", action="store_true")
    f.add_argument("--skip", action="store_true")
    f.add_argument("--tile", default=None)
    i = sub.add_parser("ising")
    i.add_argument("L", type=int)
    i.add_argument("n_lattices", type=int)
    u = sub.add_parser("fused")
    u.add_argument("gen", choices=sorted(P.GEN_IDS))
    u.add_argument("L", type=int)
    u.add_argument("n_streams", type=int)
    for q in (f, i, u):
        q.add_argument("--luxury", type=int, default=223)
        q.add_argument("--reps", type=int, default=3, help="untimed calls before the timed ones")
        q.add_argument("--timed", type=int, default=1, help="timed calls")
    a = ap.parse_args(argv)
    B.build()
    P.lib()
    tune.load_and_apply()
    h = None
    if a.what == "fill":
        if a.tile:
            P.prng_set_tile(a.gen, a.luxury if a.gen == "ranlux" else 0, *map(int, a.tile.split(",")))
        n = a.n_streams * a.n_per
        tdt = {"f32": torch.float32, "f64": torch.float64}.get(a.dtype, torch.int32)
        out = None if a.skip else torch.empty(n, dtype=tdt, device="cuda")
        if a.jump:
            fj = P.prng_fill_jump_f32 if a.dtype == "f32" else P.prng_fill_jump_u32
            call = lambda: fj(a.gen, JX0[a.gen], n, a.n_streams, out)
        else:
            h = P.prng_create(a.gen, SEED, a.n_streams, a.luxury)
            fill = {"f32": P.prng_fill_f32, "f64": P.prng_fill_f64}.get(a.dtype, P.prng_fill_u32)
            call = (lambda: P.prng_skip(h, a.n_per)) if a.skip else (lambda: fill(h, out, a.n_per))
        what = (f"{a.gen} {a.dtype} {a.n_streams}x{a.n_per}{' jump' if a.jump else ''}"
                f"{' skip' if a.skip else ''}")
        unit = lambda ms: (f"{n / ms / 1e9:.3f} T/s  "
                           f"{0.0 if a.skip else out.element_size() * n / ms / 1e6:.0f} GB/s")
    elif a.what == "ising":
        t4, t8 = P.prng_ising_thresholds(0.4406868)
        g = torch.Generator(device="cuda").manual_seed(1)
        lat = [torch.ones((a.L, a.L), dtype=torch.int8, device="cuda") for _ in range(a.n_lattices)]
        draws = [torch.randint(-2**31, 2**31 - 1, (a.L * a.L // 2,), dtype=torch.int32,
                               device="cuda", generator=g) for _ in range(a.n_lattices)]
        # descriptor rows built once in the library's struct layout, so a
        # timed launch carries no per-lattice host work
        reqs = np.zeros(a.n_lattices, P.ISING_REQ_DTYPE)
        for k, (sp, d) in enumerate(zip(lat, draws)):
            reqs[k] = (sp.data_ptr(), d.data_ptr(), a.L, 0, 8, t4, t8, 0, 0)
        call = lambda: P.prng_ising_half_sweep(reqs)
        sites = a.n_lattices * a.L * a.L // 2
        what = f"ising half-sweep {a.n_lattices} x L={a.L}"
        unit = lambda ms: f"{sites / ms / 1e6:.1f} G site updates/s"
    else:
        t4, t8 = P.prng_ising_thresholds(0.4406868)
        h = P.prng_create(a.gen, SEED, a.n_streams, a.luxury)
        spins = torch.ones((a.L, a.L), dtype=torch.int8, device="cuda")
        col = [0]

        def call():
            P.prng_ising_fused(h, spins, a.L, col[0], t4, t8)
            col[0] ^= 1
        sites = a.L * a.L // 2
        what = f"fused half-sweep {a.gen} L={a.L} on {a.n_streams} streams"
        unit = lambda ms: f"{sites / ms / 1e6:.1f} G site updates/s"
    for _ in range(a.reps):
        call()
    torch.cuda.synchronize()
    for _ in range(a.timed):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(f"{what}: {ms:.4f} ms  {unit(ms)}")
    if h is not None:
        P.prng_destroy(h)


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "kernel":
        kernel_main(sys.argv[2:])
        return
    if len(sys.argv) > 1 and sys.argv[1] == "serving":
        serving_main(sys.argv[2:])
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample", type=int, default=2**26)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-requests", type=int, default=20000)
    ap.add_argument("--batch-passes", type=int, default=3)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[1000.0, 2000.0, 4000.0, 16000.0])
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-arms", nargs="+", default=["continuous", "queue"])
    ap.add_argument("--serve-hpt", type=int, default=4)
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
