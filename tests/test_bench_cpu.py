"""The benchmark's host-side bookkeeping, without a GPU: the step's workload
matches the roofline bulk-fill configuration (2^30 u32 and 2^30 f32 per
generator, 131,072 streams x 8192 and MT19937 8192 x 131,072, two jump
fills of 2^30), and the algorithmic bytes per launch are 4 B per output
plus one read and one write of the state, per generator."""
import json

import pytest

import bench

GIB = 2**30


def test_step_is_the_roofline_configuration():
    items = bench.step_items()
    assert len(items) == 14
    assert len({lab for lab, *_ in items}) == 14
    for g in bench.GENS:
        ns, nper = bench.shape(g)
        assert ns * nper == GIB
        assert (ns, nper) == ((8192, 131072) if g == "mt19937" else (131072, 8192))
        assert (f"{g}_u32", g, "u32", GIB) in items and (f"{g}_f32", g, "f32", GIB) in items
    assert ("ggl_jump", "ggl", "jump", GIB) in items
    assert ("ranecu_jump", "ranecu", "jump", GIB) in items
    assert bench.numbers_per_step() == 14 * GIB
    assert bench.JUMP_X0 == {"ggl": 1, "ranecu": 1 | (1 << 32)}   # x0 = 1 (both components)


@pytest.mark.parametrize("gen,state_bytes_per_stream",
                         [("ggl", 4), ("xor128", 16), ("ranecu", 8), ("ranmar", 4 * 98),
                          ("ranlux", 4 * 25), ("mt19937", 4 * 624)])
def test_algorithmic_bytes_per_launch(gen, state_bytes_per_stream):
    ns, _ = bench.shape(gen)
    got = bench.algorithmic_bytes(f"{gen}_u32", gen, "u32", GIB)
    assert got == 4 * GIB + 2 * state_bytes_per_stream * ns
    # per number: 4 B + 2 * state / n_per_stream, the per-generator figures
    per_number = got / GIB
    assert 4.0 < per_number < 4.11
    assert bench.algorithmic_bytes(f"{gen}_jump", gen, "jump", GIB) == 4 * GIB


def test_recorded_traffic_needs_matching_sources_and_tile(tmp_path, monkeypatch):
    assert bench.recorded_traffic("no_such_label", "ggl") is None
    h = bench.kernel_sources_hash("ggl")
    assert len(h) == 16 and h != bench.kernel_sources_hash("mt19937")
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"per_launch": {
        "ggl_u32": {"bytes": 123, "sources": h, "tile": [128, 128, 1]},
        "mt19937_u32": {"bytes": 456, "sources": "0" * 16, "tile": [32, 624, 2]}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda g: h)
    assert bench.recorded_traffic("ggl_u32", "ggl", [128, 128, 1]) == 123
    assert bench.recorded_traffic("ggl_u32", "ggl", (128, 128, 1)) == 123
    assert bench.recorded_traffic("ggl_u32", "ggl", [128, 32, 1]) is None     # other tile
    assert bench.recorded_traffic("mt19937_u32", "mt19937", [32, 624, 2]) is None  # other sources


def test_rank_partitions():
    for g in bench.GENS:
        assert bench.rank_seed_base(g, 0) == bench.SEED
        assert bench.rank_seed_base(g, 3) - bench.rank_seed_base(g, 2) == bench.shape(g)[0]
    assert bench.rank_jump_first(0) == 0 and bench.rank_jump_first(5) == 5 * bench.JUMP_N


def test_source_hash_follows_code_not_comments():
    a = "int f(int x) {  // add one\n  return x + 1; /* plain */\n}\n"
    b = "int f(int x) {\n  /* a different\n     comment */ return x + 1;\n}  // end\n"
    c = "int f(int x) { return x + 2; }\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
