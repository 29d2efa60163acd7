"""Host-side bookkeeping of bench.py, on CPU: the source digest that retires recorded ncu traffic
when a kernel's code changes (and only then), the lookup of that traffic, and the algorithmic
bytes per kernel kind that the roofline's `achieved` is computed from."""

import os
import shutil

import pytest

import bench

FILES = ("peel.cu", "batch.cu", "peel_core.cuh", "device.cuh", "internal.h")


@pytest.fixture()
def tree(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2606_07148_gb300", "csrc")
    dst = tmp_path / "paper_2606_07148_gb300" / "csrc"
    dst.mkdir(parents=True)
    for fn in FILES:
        shutil.copy(os.path.join(src, fn), dst / fn)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_digest_ignores_comments_and_blank_lines_only(tree):
    d0 = bench.source_digest()
    p = tree / "paper_2606_07148_gb300" / "csrc" / "peel_core.cuh"
    text = p.read_text()
    p.write_text("// a new comment line\n\n" + text.replace("namespace abc {", "namespace abc {  // trailing note", 1))
    assert bench.source_digest() == d0
    p.write_text(text.replace("constexpr int ILP = 4;", "constexpr int ILP = 8;", 1))
    assert "constexpr int ILP = 4;" in text and bench.source_digest() != d0


def test_traffic_is_reported_only_for_the_recorded_digest(tree):
    dig = bench.source_digest()
    (tree / "profiles" / "dram_traffic.txt").write_text(
        "# kernel workload bytes digest\n"
        "k_cascade peel-x 48100000 %s\n"
        "k_batch batch-y 219000000000 0000000000000000\n" % dig)
    assert bench.traffic_from_profiles("k_cascade", "peel-x") == 48100000.0
    assert bench.traffic_from_profiles("k_batch", "batch-y") is None  # taken on other code
    assert bench.traffic_from_profiles("k_init", "peel-x") is None  # never recorded


def test_algorithmic_bytes_per_kernel_kind():
    # the survey's per-unit figures: 8 B offsets + 4 B count per scanned vertex, 1 B mask per
    # vertex, 16 B offsets + 8 B queue per removed vertex, 4 B per entry, 8 B per decrement,
    # 4 B per frontier check; everything else the design moves is overhead, kept apart
    st = dict(init_vertices=10, search_probes=7, stream_entries=100, stream_decrements=40,
              scanned=20, decrements=70, items=5, entries=50, pushes=6, emit_gathered=64,
              emit_scattered=0, mask_zeroed=0, round0_rows=2)
    alg, over = bench.algorithmic_bytes(st)
    assert alg[0] == 12 * 10 + 4 * 7 and over[0] == 4 * 10 + 28 * 7
    assert alg[1] == 4 * 100 + 8 * 40 + 4 * 20 + 24 * 2 and over[1] == 8 * 2
    # cascade: the 6 - 2 vertices its queue carried, its entries, its own decrements (70 - 40),
    # and one mask byte per vertex; overhead: queue bytes beyond 24 B a removed vertex, the
    # gather's id and bitmap reads (4.25 B a vertex) and the removal bits (8 B a removal)
    assert alg[2] == 24 * 4 + 4 * 50 + 8 * 30 + 64
    assert over[2] == (36 * 5 - 24 * 4) + 4.25 * 64 + 8 * 4
    # a scatter: 4 B of count per candidate, and the survivor bitmap read and cleared by the
    # expansion that writes the 64 mask bytes (1/8 B each way per vertex)
    st.update(emit_gathered=0, emit_scattered=9, mask_zeroed=64)
    alg, over = bench.algorithmic_bytes(st)
    assert alg[2] == 24 * 4 + 4 * 50 + 8 * 30 + 64
    assert over[2] == (36 * 5 - 24 * 4) + 4 * 9 + 64 / 4


def test_sampled_grid_pairs_cover_corners_and_chain_ends():
    import synth
    grid = synth.grid_pairs(8, 1, 1024)
    s8 = bench.sampled_grid_pairs(grid, 8)
    assert s8[:4] == [(1, 1), (1, 1024), (1024, 1), (1024, 1024)] and len(set(s8)) == 8
    g16 = synth.grid_pairs(16, 1, 512)
    s = bench.sampled_grid_pairs(g16, 36)
    # every chain's first and last beta, and nothing outside the grid
    for a in sorted({p[0] for p in g16}):
        assert (a, 1) in s and (a, 512) in s
    assert set(s) <= set(g16) and len(s) == 36 and len(set(s[:32])) == 32
