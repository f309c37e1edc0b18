"""Host logic of the benchmark's DRAM-traffic record (CPU).

`roofline.traffic` comes from a committed ncu capture and must be reported only
while the kernel code and the workload are the captured ones: an edit of the
full-block kernel's code (not of a comment, not of the host launchers after it)
or any other workload turns it into null.
"""
import os
import shutil

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CAPTURED = "n_mol:4096,eps:1e-05,precision:mixed,clusters:1,steps:5,warmup:3"
SRC = os.path.join("paper_1402_2880_gb300", "csrc", "k_rotate.cu")
REC = os.path.join("profiles", "dram_traffic_apply_ortho_water4096_mixed.md")


def _copy_tree(tmp_path, edit=None):
    for rel in (SRC, REC):
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), dst)
    if edit is not None:
        p = tmp_path / SRC
        p.write_text(edit(p.read_text()))
    return str(tmp_path)


def test_record_matches_the_committed_kernel():
    v = bench.measured_traffic("apply_ortho", CAPTURED)
    assert v is not None and v > 1e9


def test_other_workloads_and_launchers_get_none():
    assert bench.measured_traffic("apply_ortho", CAPTURED.replace("steps:5", "steps:2")) is None
    assert bench.measured_traffic("apply_ortho", CAPTURED.replace("mixed", "fp64")) is None
    assert bench.measured_traffic("apply_rot", CAPTURED) is None


def test_comment_and_launcher_edits_keep_the_record(tmp_path):
    def edit(src):
        src = src.replace("// Blocks between full groups", "// (edited comment)\n// Blocks between full groups", 1)
        return src + "\n// a host-side edit after the kernels\nstatic int unused_after_kernels = 0;\n"
    root = _copy_tree(tmp_path, edit)
    assert bench.measured_traffic("apply_ortho", CAPTURED, root=root) is not None


def test_kernel_code_edit_drops_the_record(tmp_path):
    def edit(src):
        key = "constexpr int kFullBatch = 8;"
        assert key in src
        return src.replace(key, "constexpr int kFullBatch = 4;", 1)
    root = _copy_tree(tmp_path, edit)
    assert bench.measured_traffic("apply_ortho", CAPTURED, root=root) is None
