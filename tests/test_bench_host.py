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
    st = dict(init_vertices=10, search_probes=7, stream_entries=100, stream_decrements=40,
              scanned=20, decrements=70, items=5, entries=50, pushes=6, emit_gathered=64,
              emit_scattered=0)
    b = bench.algorithmic_bytes(st)
    assert b[0] == 16 * 10 + 4 * 7
    assert b[1] == 4 * 100 + 8 * 40 + 4 * 20
    # cascade: items, entries, its own decrements (70 - 40), push slots, the gather (5.25 B a
    # vertex) and the removal bits (8 B a push)
    assert b[2] == 28 * 5 + 4 * 50 + 8 * 30 + 8 * 6 + 5.25 * 64 + 8 * 6
    st.update(emit_gathered=0, emit_scattered=9)
    assert bench.algorithmic_bytes(st)[2] == 28 * 5 + 4 * 50 + 8 * 30 + 8 * 6 + 4 * 9
