"""The bench line's `roofline.traffic` is the DRAM traffic ncu measured for
the step kernel, recorded with a hash of the kernel's sources; the bench
reports it only while the sources still hash the same.  The hash ignores
comments and whitespace and changes with any code token."""
import os
import shutil

import bench

FILES = ("step2d.cuh", "common.cuh", "limiter.cuh", "tables.cuh")


def _copy_tree(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2307_06471_gb300", "csrc")
    dst = tmp_path / "paper_2307_06471_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in FILES:
        shutil.copy(os.path.join(src, f), dst / f)
    return dst


def test_hash_follows_code_not_comments(tmp_path, monkeypatch):
    dst = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_src_hash()
    assert h0 == bench.kernel_src_hash()
    p = dst / "limiter.cuh"
    text = p.read_text()
    # a comment (line and block) and a change of indentation: same hash
    p.write_text("// a note\n/* a block\n   comment */\n" + text.replace("\n    ", "\n        ", 3))
    assert bench.kernel_src_hash() == h0
    # one code token changed: another hash
    assert "T(0.5)" in text
    p.write_text(text.replace("T(0.5)", "T(0.25)", 1))
    assert bench.kernel_src_hash() != h0


def test_recorded_traffic_is_a_launch_of_the_workload():
    """The record is one launch's read + write bytes: below the algorithmic
    192 bytes per cell (u^n read, u^{n+1} written) of the 1920 x 480 mesh,
    as part of u^{n+1} is still in L2 when the kernel ends, and above the
    read of u^n alone."""
    t = bench.TRAFFIC
    assert set(t) == {"bytes", "src_hash"} and len(t["src_hash"]) == 16
    cells = 1920 * 480
    assert 96 * cells < t["bytes"] < 192 * cells
