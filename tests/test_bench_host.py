"""Host logic of bench.py that decides what the JSON line reports: the
kernel-source hash that ties the committed ncu traffic to the code, and the
parser of that summary."""
import os
import shutil

import bench

CSRC = ("acoustic.cu", "acoustic_kernel.cuh", "ptx.cuh")


def _copy_tree(tmp_path):
    dst = tmp_path / "paper_1608_03984_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in CSRC:
        shutil.copy(os.path.join(bench.ROOT, "paper_1608_03984_gb300", "csrc", f), dst / f)
    (tmp_path / "profiles").mkdir()
    return dst


def test_source_hash_ignores_comments_but_not_code(tmp_path):
    dst = _copy_tree(tmp_path)
    h0 = bench.kernel_source_sha(str(tmp_path))
    assert h0 == bench.kernel_source_sha()
    src = (dst / "acoustic.cu").read_text()
    (dst / "acoustic.cu").write_text("// a new comment\n/* and a\n block */\n" + src.replace("\n", "\n\n"))
    assert bench.kernel_source_sha(str(tmp_path)) == h0
    (dst / "acoustic.cu").write_text(src.replace("return 1;", "return 2;", 1))
    assert bench.kernel_source_sha(str(tmp_path)) != h0


def test_traffic_summary_is_used_only_for_the_matching_source(tmp_path):
    _copy_tree(tmp_path)
    sha = bench.kernel_source_sha(str(tmp_path))
    body = "TRAFFIC_BYTES_PER_POINT order=2 16.25\nTRAFFIC_BYTES_PER_POINT order=16 16.5\n"
    summary = tmp_path / "profiles" / "acoustic_step_592_dram.md"
    summary.write_text(body + "source_sha=%s\n" % sha)
    assert bench.ncu_traffic_per_point(str(tmp_path)) == {2: 16.25, 16: 16.5}
    summary.write_text(body + "source_sha=%s\n" % ("0" * 16))
    assert bench.ncu_traffic_per_point(str(tmp_path)) is None
    summary.unlink()
    assert bench.ncu_traffic_per_point(str(tmp_path)) is None


def test_closure_operating_point():
    """The largest k whose field error stays within 5% of the every-step
    closure's; k = 1 when no sub-cycled run qualifies."""
    ms = {"fine": 1000.0, "closure": 1000.0}
    sub = {"2": {"error_vs_fine": {"field": 0.0101}, "speedup_vs_fine": 1.9},
           "4": {"error_vs_fine": {"field": 0.0104}, "speedup_vs_fine": 3.4},
           "8": {"error_vs_fine": {"field": 0.0300}, "speedup_vs_fine": 5.6}}
    op = bench.operating_point(0.0100, ms, sub)
    assert op == {"every": 4, "field_error": 0.0104, "speedup_vs_fine": 3.4}
    bad = {k: {"error_vs_fine": {"field": 0.05}, "speedup_vs_fine": 9.0} for k in ("2", "4")}
    assert bench.operating_point(0.0100, ms, bad)["every"] == 1
