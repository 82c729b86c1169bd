"""The multi-GPU benchmark path's host logic on CPU, as two gloo ranks on
127.0.0.1 (no GPU, no NCCL).  Per rank: its streams, seeded from
bench.rank_seed_base, are streams [r n, (r + 1) n) of one handle of 2 n
streams (checked with the oracle on sampled streams); its jump fills cover
the next N draws of the one sequence after the previous rank's; the timing reduction
returns the slowest rank's time on every rank; the reference arm prints its
JSON line from rank 0 only."""
import argparse
import contextlib
import io
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

WORLD = 2


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    out = {"rank": rank}
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import bench
        import oracle
        pos = np.array([0, 1, 2, 999], dtype=np.uint64)
        checks = []
        for g in bench.GENS:
            n = bench.shape(g)[0]
            base = bench.rank_seed_base(g, rank)
            lux = bench.RANLUX_P if g == "ranlux" else 0
            for i in (0, 1, n - 1):
                mine = oracle.sample(g, base, i, pos, luxury=lux)
                glob = oracle.sample(g, bench.SEED, rank * n + i, pos, luxury=lux)
                checks.append(bool(np.array_equal(mine, glob)))
        out["partition_ok"] = all(checks)
        out["jump_first"] = bench.rank_jump_first(rank)
        out["bases"] = {g: bench.rank_seed_base(g, rank) for g in bench.GENS}
        out["max_ms"] = bench.max_over_ranks(10.0 + rank, dist, "cpu")
        buf = io.StringIO()
        args = argparse.Namespace(cpu_sample=1 << 12, warmup=0, steps=1)
        with contextlib.redirect_stdout(buf):
            bench.run_reference(args, rank, world)
        out["printed"] = buf.getvalue()
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, which fails the test
        out["error"] = repr(e)
    q.put(out)


def test_two_gloo_ranks_partition_reduce_and_print():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    try:
        res = sorted((q.get(timeout=300) for _ in procs), key=lambda d: d["rank"])
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    for r in res:
        assert "error" not in r, r.get("error")
        assert r["partition_ok"]
        assert r["max_ms"] == 10.0 + (WORLD - 1)
    import bench
    for g in bench.GENS:   # disjoint, adjacent stream ranges
        assert res[1]["bases"][g] - res[0]["bases"][g] == bench.shape(g)[0]
    # jump fills: rank r covers draws [r N, (r + 1) N) of the one sequence
    assert res[0]["jump_first"] == 0 and res[1]["jump_first"] == bench.JUMP_N
    assert res[1]["printed"] == ""
    lines = [l for l in res[0]["printed"].splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == WORLD
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
