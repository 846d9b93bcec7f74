"""bench.py takes a kernel's DRAM traffic and instruction count from its
committed ncu summary only when that summary was taken on the kernel's
current source (a hash of the files it is built from) and, when the summary
names one, on the schedule being benchmarked; otherwise the line carries
null. These tests build summaries in a temporary tree and check each case,
and check the algorithmic bytes per step the roofline uses (49.1 B per point
at 128x128x80). No GPU."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SCHED = {"fusion": 1, "staging": 0, "tile_i": 32, "tile_j": 16, "unroll": 2, "k_chunk": 2, "arith": 2,
         "sweep": 0, "slabs": 0}


@pytest.fixture
def tree(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2005_13014_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "a.cu").write_text("kernel a\n")
    (csrc / "b.cuh").write_text("header b\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _kernel(profile="k.md"):
    return {"name": "k", "src": ["a.cu", "b.cuh"], "profile": profile}


def _write(tree, sha, sched=None, traffic=1234, instr=99):
    text = f"# k\n\nkernel_source_sha256_16: {sha}\ndram_bytes_per_launch: {traffic}\n"
    if sched is not None:
        import json
        text += f"captured_schedule: {json.dumps(sched)}\n"
    text += f"warp_instructions_per_launch: {instr}\n"
    (tree / "profiles" / "k.md").write_text(text)


def test_current_source_and_schedule(tree):
    _write(tree, bench._kernel_source_hash(["a.cu", "b.cuh"]), SCHED)
    assert bench._ncu_traffic(_kernel(), SCHED) == 1234
    assert bench._ncu_figure(_kernel(), "warp_instructions_per_launch", SCHED) == 99


def test_changed_source_gives_null(tree):
    _write(tree, bench._kernel_source_hash(["a.cu", "b.cuh"]), SCHED)
    (tree / "paper_2005_13014_gb300" / "csrc" / "b.cuh").write_text("header b, edited\n")
    assert bench._ncu_traffic(_kernel(), SCHED) is None


def test_other_schedule_gives_null(tree):
    _write(tree, bench._kernel_source_hash(["a.cu", "b.cuh"]), SCHED)
    assert bench._ncu_traffic(_kernel(), dict(SCHED, k_chunk=4)) is None
    assert bench._ncu_traffic(_kernel(), dict(SCHED, tile_j=8)) is None


def test_summary_without_schedule_serves_any(tree):
    _write(tree, bench._kernel_source_hash(["a.cu", "b.cuh"]), None)
    assert bench._ncu_traffic(_kernel(), dict(SCHED, k_chunk=4)) == 1234


def test_missing_summary_gives_null(tree):
    assert bench._ncu_traffic(_kernel("absent.md"), SCHED) is None
    assert bench._ncu_traffic(_kernel(None), SCHED) is None


def test_algorithmic_bytes_per_step():
    """u and v over their i/j halo of 2, w with its i+1 column, coeff and the
    two outputs over the domain, 8 bytes each: 64,327,680 B at 128x128x80."""
    n = (128, 128, 80)
    total = sum(bench._field_bytes(f, n) for f in ("u", "v", "w", "coeff", "u_out", "v_out"))
    assert total == 2 * 132 * 132 * 80 * 8 + 129 * 128 * 80 * 8 + 3 * 128 * 128 * 80 * 8 == 64327680


def test_headline_kernels_name_their_summaries():
    ks = bench._kernels_of(SCHED)
    assert [k["name"] for k in ks] == ["hdiff_fixed_kernel", "hv_thomas_kernel"]
    for k in ks:
        assert k["profile"] and os.path.exists(os.path.join(ROOT, "profiles", k["profile"]))
