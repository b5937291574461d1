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
    summary = tmp_path / "profiles" / bench.TRAFFIC_SUMMARY
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
    assert op == {"every": 4, "field_error": 0.0104, "speedup_vs_fine": 3.4, "selected_on": "evaluation models"}
    bad = {k: {"error_vs_fine": {"field": 0.05}, "speedup_vs_fine": 9.0} for k in ("2", "4")}
    assert bench.operating_point(0.0100, ms, bad)["every"] == 1


def test_closure_operating_point_chosen_on_validation_models():
    """With validation errors, k is chosen on them and the evaluation
    models' error and speed-up at that k are reported."""
    ms = {"fine": 1000.0, "closure": 1000.0}
    sub = {"2": {"error_vs_fine": {"field": 0.0101}, "speedup_vs_fine": 1.9},
           "4": {"error_vs_fine": {"field": 0.0104}, "speedup_vs_fine": 3.4},
           "8": {"error_vs_fine": {"field": 0.0300}, "speedup_vs_fine": 5.6}}
    val = {"closure": 0.020, "every": {"2": 0.0201, "4": 0.0250, "8": 0.0600}, "label": "validation models 1, 2"}
    op = bench.operating_point(0.0100, ms, sub, val)
    assert op == {"every": 2, "field_error": 0.0101, "speedup_vs_fine": 1.9,
                  "selected_on": "validation models 1, 2"}
    val["every"] = {"2": 0.03, "4": 0.04, "8": 0.05}
    op = bench.operating_point(0.0100, ms, sub, val)
    assert op["every"] == 1 and op["field_error"] == 0.0100 and op["speedup_vs_fine"] == 1.0


def _full_result():
    """A result of the shape run_fdwave assembles, with every section filled
    as on the benchmark (16 held-out closure models, five orders)."""
    orders = ("2", "4", "8", "12", "16")
    per_order = {o: {"kernel_ms": 0.5823, "kernel_gpts": 356.1234, "tile": 1, "zchunks": 4,
                     "achieved_gbs": 5700.12, "frac_of_measured_hbm": 0.8412345, "I_alg_paper": 2.125,
                     "paper_model_gflops": 12345.678, "roofline_gpts_paper_model": 424.1,
                     "ncu_dram_bytes_per_point": 16.3} for o in orders}
    err = {"field": 0.0153, "traces": 0.0106, "traces_by_depth": {"5": 0.0106, "10": 0.0099, "20": 0.0084}}
    per_model = [{m: dict(err) for m in ("coarse", "closure", "closure_every2", "closure_every4",
                                         "closure_every8", "closure_every16")} for _ in range(16)]
    return {
        "metric": "Gpts/s per timestep", "value": 346.123456, "unit": "Gpts/s", "n_gpus": 1, "steps": 20,
        "warmup": 5, "ms_per_step": 2.9971, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "random_acoustic 512^3 + 40-point sponge (592x592x592 computational), h=10 m, "
                               "orders 2/4/8/12/16 (one step of each per bench step), Ricker 10 Hz, "
                               "256x256 receivers", "grid": [592, 592, 592], "orders": [2, 4, 8, 12, 16],
                   "equation": "acoustic", "l2": "inputs larger than L2 (each field 830 MB)",
                   "global_batch": 5, "parallelism": "single"},
        "roofline": {"kernel": "acoustic_tma_kernel (orders 2/4/8/12/16)", "bound": "hbm",
                     "achieved": 5700.1, "peak": 6790.7, "unit": "GB/s", "frac": 0.8394, "peak_source": "measured",
                     "traffic": 3.4e9, "algorithmic_bytes_per_launch": 3319595008},
        "per_order": per_order,
        "e2e": {"value": 291.2, "unit": "Gpts/s", "h2d_bytes_per_step": 27000000, "d2h_bytes_per_step": 2621440,
                "note": "per order: model/sources/receivers uploaded from pinned host memory"},
        "cpu_baseline": {"value": 0.4156, "unit": "Gpts/s", "cores": 16, "kind": "oracle",
                         "sample": "16 x 592 x 592 slab of the 592x592x592 grid per order (orders 2/4/8/12/16), "
                                   "FP64 oracle, 12.3 s"},
        "tti": {"workload": "random_tti", "8": {st: {"kernel_ms": 1.5, "gpts": 66.7, "achieved_gbs": 2900.0,
                                                     "frac_of_measured_hbm": 0.43} for st in ("f32", "bf16", "f16")},
                "12": {st: {"kernel_ms": 2.1, "gpts": 47.2, "achieved_gbs": 2000.0, "frac_of_measured_hbm": 0.31}
                       for st in ("f32", "bf16", "f16")}},
        "storage": dict({o: {st: {"kernel_ms": 0.4, "gpts": 500.0, "speedup_vs_f32": 1.2345,
                                  "achieved_gbs": 4000.0, "frac_of_measured_hbm": 0.6}
                             for st in ("bf16", "f16")} for o in orders},
                        errors_vs_fp64_oracle={
                            "acoustic": {st: {"traces": 0.0161234, "u": 0.029} for st in ("f32", "bf16", "f16")},
                            "tti": {st: {"traces": 0.011, "p": 0.069, "r": 0.082} for st in ("f32", "bf16", "f16")},
                            "problems": "x" * 200}),
        "fwi": {"workload": "fwi 256^3", "gradient_s": 19.01, "per_shot_s": 1.19, "shots": 16, "misfit": 1.0,
                "stencil_steps": 96000, "gpts_equiv": 190.0, "gradient_finite": True},
        "closure": {"error_vs_fine": {"coarse": {"field": 0.0448, "traces": 0.0178},
                                      "closure": {"field": 0.0145, "traces": 0.0190}},
                    "speedup_vs_fine": {"coarse": 16.4, "closure": 1.01},
                    "operating_point": {"every": 4, "field_error": 0.01451234, "speedup_vs_fine": 3.4212,
                                        "selected_on": "evaluation models"},
                    "per_model": per_model, "every_k_steps": {str(k): {"x": 1} for k in (2, 4, 8, 16)}},
        "config1": {"workload": "two_layer 64^3", "ms_per_run": 2.5, "us_per_step": 12.5, "gpts": 47.4},
        "paper_model_gb300": {"table_cost": {str(o): {"I_alg": 1.0} for o in range(2, 26, 2)}},
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 40},
        "gpu_launches": 300,
    }


def test_headline_line_is_compact_and_complete():
    """The printed line carries the headline metric, roofline, e2e, CPU
    baseline, clocks and one summary per section, within a fixed byte
    budget (a long line is cut off by readers that keep only its tail)."""
    import json
    full = _full_result()
    line = bench.headline(full, "/tmp/some/dir/bench_details.json")
    text = json.dumps(line)
    assert len(text) <= bench.HEADLINE_MAX_BYTES, len(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "dtype", "config", "roofline", "e2e", "cpu_baseline", "clocks", "gpu_launches"):
        assert line[k] == (full[k] if k != "e2e" else line[k]), k
    assert line["value"] > 0 and line["roofline"]["frac"] > 0
    assert "note" not in line["e2e"] and line["e2e"]["h2d_bytes_per_step"] > 0
    assert set(line["per_order"]) == set(full["per_order"])
    assert set(line["sections"]) == {"tti", "storage_speedup_vs_f32", "storage_error_vs_fp64", "fwi", "closure",
                                     "config1"}
    assert line["sections"]["storage_error_vs_fp64"]["tti"]["bf16"]["p"] == 0.069
    assert line["sections"]["closure"]["operating_point"]["every"] == 4
    assert line["details"] == "bench_details.json"
    # sections that did not run are simply absent
    for k in ("tti", "storage", "fwi", "closure", "config1"):
        full[k] = None
    assert bench.headline(full, "d.json")["sections"] == {}


def test_launches_per_step_follows_the_sparse_kernels():
    """One fused injection + interpolation block up to 256 receivers, two
    kernels above (the stencil is the third)."""
    assert bench.launches_per_step(0) == 2
    assert bench.launches_per_step(32) == 2
    assert bench.launches_per_step(256) == 2
    assert bench.launches_per_step(257) == 3
    assert bench.launches_per_step(65536) == 3
