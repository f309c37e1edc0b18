"""Host logic of the benchmark's DRAM-traffic record (CPU).

`roofline.traffic` comes from a committed ncu capture and must be reported only
while the kernel code and the workload are the captured ones: an edit of the
sweep source's code (kernels or launchers, not comments) or of the shared
header's code, or any other workload, turns it into null. The tests write
their own record for the current code into a copy of the tree.
"""
import os
import shutil

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORKLOAD = "n_mol:4096,eps:1e-05,precision:mixed,clusters:1,replayed_iteration:4"
SRC = os.path.join("paper_1402_2880_gb300", "csrc", "k_rotate.cu")
HDR = os.path.join("paper_1402_2880_gb300", "csrc", "sscf_internal.h")
REC = os.path.join("profiles", "dram_traffic_apply_ortho_water4096_mixed.md")


def _tree(tmp_path, edit=None, edit_header=None):
    """A copy of the kernel source and header with a record of their current
    code, then (optionally) one of them edited."""
    src = tmp_path / SRC
    src.parent.mkdir(parents=True, exist_ok=True)
    shutil.copy(os.path.join(ROOT, SRC), src)
    hdr = tmp_path / HDR
    shutil.copy(os.path.join(ROOT, HDR), hdr)
    rec = tmp_path / REC
    rec.parent.mkdir(parents=True, exist_ok=True)
    digest = bench.kernel_code_digest(str(src))
    rec.write_text("# capture\n\ntraffic: apply_ortho bytes_per_call=123456789 "
                   f"kernel_code_sha256={digest} workload={WORKLOAD}\n")
    if edit is not None:
        src.write_text(edit(src.read_text()))
    if edit_header is not None:
        hdr.write_text(edit_header(hdr.read_text()))
    return str(tmp_path)


def test_record_of_the_current_code_is_reported(tmp_path):
    assert bench.measured_traffic("apply_ortho", WORKLOAD, root=_tree(tmp_path)) == 123456789.0


def test_other_workloads_and_launchers_get_none(tmp_path):
    root = _tree(tmp_path)
    assert bench.measured_traffic("apply_ortho", WORKLOAD.replace("iteration:4", "iteration:6"), root=root) is None
    assert bench.measured_traffic("apply_ortho", WORKLOAD.replace("mixed", "fp64"), root=root) is None
    assert bench.measured_traffic("apply_rot", WORKLOAD, root=root) is None


def test_comment_edits_keep_the_record(tmp_path):
    def edit(src):
        return src.replace("// Blocks between full groups", "// (edited comment)\n// Blocks between full groups", 1)
    assert bench.measured_traffic("apply_ortho", WORKLOAD, root=_tree(tmp_path, edit)) == 123456789.0


def test_kernel_code_edit_drops_the_record(tmp_path):
    def edit(src):
        key = "constexpr int kFullBatch = 8;"
        assert key in src
        return src.replace(key, "constexpr int kFullBatch = 4;", 1)
    assert bench.measured_traffic("apply_ortho", WORKLOAD, root=_tree(tmp_path, edit)) is None


def test_launcher_edit_drops_the_record(tmp_path):
    def edit(src):
        key = "const int chunks = (c->n_mol + kFullCH - 1) / kFullCH;"
        assert key in src
        return src.replace(key, "const int chunks = (c->n_mol + 2 * kFullCH - 1) / kFullCH;", 1)
    assert bench.measured_traffic("apply_ortho", WORKLOAD, root=_tree(tmp_path, edit)) is None


def test_shared_header_edit_drops_the_record(tmp_path):
    def edit(src):
        key = "constexpr int kOrthoCap = 48 * 48;"
        assert key in src
        return src.replace(key, "constexpr int kOrthoCap = 48 * 49;", 1)
    assert bench.measured_traffic("apply_ortho", WORKLOAD, root=_tree(tmp_path, edit_header=edit)) is None


def test_committed_record_is_well_formed():
    rec = os.path.join(ROOT, "profiles", "dram_traffic_apply_ortho_water4096_mixed.md")
    with open(rec) as f:
        line = next(l for l in f if l.startswith("traffic: apply_ortho "))
    fields = dict(kv.split("=", 1) for kv in line.split()[2:])
    assert float(fields["bytes_per_call"]) > 1e9
    assert len(fields["kernel_code_sha256"]) == 64
    assert fields["workload"].startswith("n_mol:4096,eps:1e-05,precision:mixed,clusters:1,replayed_iteration:")
