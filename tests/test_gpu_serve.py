"""The serving loop: every result -- in the mix, served with continuous
batching -- equals the oracle's and what the client gets alone."""
import numpy as np
import pytest

import oracle
from paper_1003_1898_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1003_1898_gb300 as P  # noqa: E402
from paper_1003_1898_gb300 import serve  # noqa: E402

NS = 64          # streams per client: divides L*L/2 for L in 32, 64, 128


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_1898_gb300 import build
    build.build()
    P.lib()


def _requests(n, clients, rate, seed):
    raw = W.serving_requests(n, rate, n_clients=clients, seed=seed, fill_min=10, fill_max=5000,
                             ising_sizes=(32, 64, 128), sweeps=3)
    return [serve.Request(**r) for r in raw]


def _results(reqs):
    out = {}
    for r in reqs:
        out[r.rid] = (r.out.cpu().numpy().reshape(-1)[:r.n].view(np.uint32) if r.kind == "fill"
                      else r.spins.cpu().numpy())
    return out


@pytest.mark.parametrize("hpt", [1, 3, 4])
def test_mix_equals_oracle_and_clients_alone(hpt):
    # hpt: Ising half-sweeps per tick (3: one fill of three half-sweeps' draws,
    # read as column blocks of the stream rows, and three launches).
    specs = W.serving_clients(12, seed=99)
    reqs = _requests(80, 12, 1e9, seed=7)
    srv = serve.Server(specs, n_streams=NS, keep_results=True, half_sweeps_per_tick=hpt)
    try:
        done = srv.run(reqs, realtime=False)
    finally:
        srv.close()
    mixed = _results(done)
    # oracle: each client's requests in arrival order, its streams advancing
    consumed = {}
    for r in sorted(done, key=lambda r: (r.arrival, r.rid)):
        g, lux, seed = specs[r.client]
        skip = consumed.get(r.client, 0)
        if r.kind == "fill":
            per = srv.fill_shape(r.n)[0]
            ref = oracle.fill(g, seed, NS, per, luxury=lux, skip=skip).reshape(-1)[:r.n]
            if r.f32:
                ref = oracle.to_f32(g, ref).view(np.uint32)
            np.testing.assert_array_equal(mixed[r.rid], ref, err_msg=f"fill {r.rid}")
            consumed[r.client] = skip + per
        else:
            lat, _ = oracle.ising_run(g, seed, NS, r.L, r.sweeps, luxury=lux, skip=skip)
            np.testing.assert_array_equal(mixed[r.rid], lat, err_msg=f"ising {r.rid}")
            consumed[r.client] = skip + r.sweeps * r.L * r.L // NS
    # each client alone, in its own server, gives the same bytes
    for c in sorted({r.client for r in done})[:4]:
        mine = [serve.Request(rid=r.rid, client=0, kind=r.kind, arrival=r.arrival, n=r.n,
                              f32=r.f32, L=r.L, sweeps=r.sweeps) for r in done if r.client == c]
        alone_srv = serve.Server([specs[c]], n_streams=NS, keep_results=True)   # one per tick
        try:
            alone = _results(alone_srv.run(mine, realtime=False))
        finally:
            alone_srv.close()
        for rid, v in alone.items():
            np.testing.assert_array_equal(v, mixed[rid])


def test_realtime_arrivals_complete_with_same_results():
    specs = W.serving_clients(8, seed=5)
    reqs_a = _requests(60, 8, 3000.0, seed=11)
    reqs_b = _requests(60, 8, 3000.0, seed=11)
    s1 = serve.Server(specs, n_streams=NS, keep_results=True)
    s2 = serve.Server(specs, n_streams=NS, keep_results=True)
    try:
        a = s1.run(reqs_a, realtime=True)
        b = s2.run(reqs_b, realtime=False)
    finally:
        s1.close()
        s2.close()
    ra, rb = _results(a), _results(b)
    for rid in ra:
        np.testing.assert_array_equal(ra[rid], rb[rid])
    st = serve.latency_stats(a)
    assert st["requests"] == 60 and st["p50_ms"] >= 0 and st["p99_ms"] >= st["p50_ms"]
    assert all(r.done >= r.arrival for r in a)


def test_memory_cap_defers_admission():
    specs = W.serving_clients(4, seed=1)
    reqs = [serve.Request(rid=i, client=i % 4, kind="ising", L=128, sweeps=2) for i in range(8)]
    state = 0
    srv = serve.Server(specs, n_streams=NS, mem_cap=1, keep_results=True)
    try:
        state = srv.mem_state
        srv.mem_cap = state + srv.request_bytes(reqs[0]) + 1   # room for one lattice at a time
        done = srv.run(reqs, realtime=False)
    finally:
        srv.close()
    assert all(r.done is not None for r in done)
    # one at a time: completion times strictly increase
    t = sorted(r.done for r in done)
    assert all(b > a for a, b in zip(t, t[1:]))
