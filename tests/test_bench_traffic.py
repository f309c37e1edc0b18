"""Host logic of the benchmark's DRAM-traffic record (CPU).

`roofline.traffic` comes from a committed ncu capture and must be reported only
while the kernel code and the workload are the captured ones: an edit of the
full-block kernel's code (not of a comment, not of the host launchers after it)
or any other workload turns it into null. The tests write their own record for
the current kernel code into a copy of the tree.
"""
import os
import shutil

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORKLOAD = "n_mol:4096,eps:1e-05,precision:mixed,clusters:1,steps:5,warmup:3"
SRC = os.path.join("paper_1402_2880_gb300", "csrc", "k_rotate.cu")
REC = os.path.join("profiles", "dram_traffic_apply_ortho_water4096_mixed.md")


def _tree(tmp_path, edit=None):
    """A copy of the kernel source with a record of its current code, then
    (optionally) the source edited."""
    src = tmp_path / SRC
    src.parent.mkdir(parents=True, exist_ok=True)
    shutil.copy(os.path.join(ROOT, SRC), src)
    rec = tmp_path / REC
    rec.parent.mkdir(parents=True, exist_ok=True)
    digest = bench.kernel_code_digest(str(src))
    rec.write_text("# capture\n\ntraffic: apply_ortho bytes_per_call=123456789 "
                   f"kernel_code_sha256={digest} workload={WORKLOAD}\n")
    if edit is not None:
        src.write_text(edit(src.read_text()))
    return str(tmp_path)


def test_committed_record_is_well_formed():
    with open(os.path.join(ROOT, REC)) as f:
        line = next(l for l in f if l.startswith("traffic: apply_ortho "))
    fields = dict(kv.split("=", 1) for kv in line.split()[2:])
    assert float(fields["bytes_per_call"]) > 1e9
    assert len(fields["kernel_code_sha256"]) == 64
    assert fields["workload"] == WORKLOAD


def test_record_of_the_current_code_is_reported(tmp_path):
    assert bench.measured_traffic("apply_ortho", WORKLOAD, root=_tree(tmp_path)) == 123456789.0


def test_other_workloads_and_launchers_get_none(tmp_path):
    root = _tree(tmp_path)
    assert bench.measured_traffic("apply_ortho", WORKLOAD.replace("steps:5", "steps:2"), root=root) is None
    assert bench.measured_traffic("apply_ortho", WORKLOAD.replace("mixed", "fp64"), root=root) is None
    assert bench.measured_traffic("apply_rot", WORKLOAD, root=root) is None


def test_comment_and_launcher_edits_keep_the_record(tmp_path):
    def edit(src):
        src = src.replace("// Blocks between full groups", "// (edited comment)\n// Blocks between full groups", 1)
        return src + "\n// a host-side edit after the kernels\nstatic int unused_after_kernels = 0;\n"
    assert bench.measured_traffic("apply_ortho", WORKLOAD, root=_tree(tmp_path, edit)) == 123456789.0


def test_kernel_code_edit_drops_the_record(tmp_path):
    def edit(src):
        key = "constexpr int kFullBatch = 8;"
        assert key in src
        return src.replace(key, "constexpr int kFullBatch = 4;", 1)
    assert bench.measured_traffic("apply_ortho", WORKLOAD, root=_tree(tmp_path, edit)) is None
