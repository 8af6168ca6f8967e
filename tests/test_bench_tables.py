"""Host logic of bench.py's measured tables (CPU).

The ncu figures (DRAM bytes and issue slots per voxel) are reported only while
the kernel code they were measured on is unchanged (else null): the gate
hashes the source without comments and blank space, so an edited comment
keeps the figures and an edited statement drops them.  The algorithmic byte model adds up to the
schedule totals the design states.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _hash_of(tmp_path, monkeypatch, text):
    d = tmp_path / "paper_2404_02813_gb300" / "csrc"
    d.mkdir(parents=True, exist_ok=True)
    (d / "k.cuh").write_text(text)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return bench._source_sha("k.cuh")


def test_hash_ignores_comments_and_blank_space(tmp_path, monkeypatch):
    base = _hash_of(tmp_path, monkeypatch, "int f(int a) {\n    return a + 1;  // one\n}\n")
    assert _hash_of(tmp_path, monkeypatch, "int f(int a) { return a + 1; }") == base
    assert _hash_of(tmp_path, monkeypatch, "/* a block\n comment */ int f(int a) {\n return a + 1; // other\n}") == base
    assert _hash_of(tmp_path, monkeypatch, "int f(int a) { return a + 2; }") != base
    assert _hash_of(tmp_path, monkeypatch, "int f(int a) { return a+1; }") != base  # code text, not semantics


@pytest.mark.parametrize("img,st,force,total", [(2, 4, "li", 72), (1, 4, "eq15", 66), (1, 2, "li", 62)])
def test_schedule_bytes(img, st, force, total):
    per = bench.algo_bytes_per_voxel(img, st, force)
    kernels = ["rsf_ta_xy", "rsf_ta_z", "rsf_tb_z"] + ([] if force == "eq15" else ["rsf_tb_xy"])
    assert sum(per[k] for k in kernels) == total
    # DRAM traffic measured by ncu sits at (or just under) the algorithmic bytes
    if img == 2 and st == 4 and force == "li":
        for k in kernels:
            assert 0.9 * per[k] <= bench.NCU_TRAFFIC[k]["bytes_per_voxel"] <= 1.02 * per[k]
