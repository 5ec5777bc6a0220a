"""Host-side logic of the benchmark's JSON line (no GPU): the equal-recall
selection picks the largest tolerance, and then the largest decision
threshold, whose recall reaches plain OPH's."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _q(oph_recall, eps_recall, thr_recall):
    q = {"oph_full_scan": {"recall": oph_recall, "precision": 0.97}, "truly_similar": 100}
    for e, r in eps_recall.items():
        q["hoph_eps_%g" % e] = {"recall": r, "precision": 0.95}
    for t, r in thr_recall.items():
        q["hoph_T_%d_%d" % t] = {"recall": r, "precision": 0.9 + t[0] / t[1] / 10}
    return q


def test_equal_recall_picks_the_largest_eps_then_the_largest_threshold():
    eps = {1e-4: 0.95, 1e-5: 0.96, 0.0: 0.97}
    thr = {(699, 1000): 0.96, (697, 1000): 0.97, (69, 100): 0.99}
    q = _q(0.97, eps, thr)
    runs_e = {e: {"ms": 0.4 + i * 0.1} for i, e in enumerate(eps)}
    runs_t = {t: {"ms": 0.45} for t in thr}
    out = bench.equal_recall(q, runs_e, 1024, 10 ** 7, 4096, runs_t)
    assert out["eps_at_equal_recall"] == 0.0
    assert out["decision_threshold_at_equal_recall"] == "697/1000"
    assert abs(out["value_at_equal_recall_by_threshold"] - 1024 * 10 ** 7 / 0.45e-3) < 1
    assert out["oph_full_scan_recall"] == 0.97


def test_equal_recall_reports_none_when_nothing_reaches_oph():
    q = _q(0.99, {1e-4: 0.95}, {(699, 1000): 0.96})
    out = bench.equal_recall(q, {1e-4: {"ms": 0.4}}, 1024, 10 ** 7, 4096,
                             {(699, 1000): {"ms": 0.4}})
    assert out["eps_at_equal_recall"] is None
    assert out["decision_threshold_at_equal_recall"] is None
    assert out["value_at_equal_recall_by_threshold"] is None


def _fake_args(**over):
    a = dict(gpus=1, steps=1000, warmup=10, rows=10_000_000, queries=1024, in_flight=8,
             decision_thr="697/1000", details=None)
    a.update(over)
    return type("A", (), a)()


def _fake_line(world=1):
    args = _fake_args()
    head = {"value": 2.8123456789e13, "ms": 366.123456789, "gpu_launches": 7000,
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0,
                       "reasons": ["sw_power_cap"], "samples": 123},
            "roofline": {"bound": "hbm", "kernel": "filter_kernel",
                         "achieved": 7171.123456789, "unit": "GB/s",
                         "traffic": 2577060000.123, "alg_bytes": 2560262144,
                         "kernel_ms": 0.35699999}}
    line = bench.headline_line(args, world, head, {"hbm_gbs": 6777.0}, "measured")
    line["e2e"] = {"value": 2.74e13, "unit": bench.UNIT, "h2d_bytes_per_step": 2029576,
                   "d2h_bytes_per_step": 65544, "ms_per_step": 0.374111}
    line["cpu_baseline"] = {"value": 8.9e7, "unit": bench.UNIT, "cores": 144, "kind": "oracle",
                            "cpu_model": "Neoverse-V2 with a fairly long model name string",
                            "value_one_core": 5.3e6,
                            "sample": "C oracle: sketch 1024 query sets + (1:2)HOPH vs rows "
                                      "0..1234567 (1264197632 pairs, 14.9 s); one core: rows "
                                      "0..1999"}
    line["metric_parts"] = bench.metric_parts({
        "sketch": {"sets_per_s": 7.5e8, "roofline": {"frac": 0.33}},
        "equal_recall": {"headline_recall": 0.9724, "oph_full_scan_recall": 0.9724,
                         "headline_at_equal_recall": True},
        "oph_full_scan_baseline": {"value": 6.5e9},
        "headline": {"value_at_T": 2.81e13}})
    return line


def test_headline_is_one_json_line_under_2kb_with_the_contract_keys():
    import json
    text = bench.headline_json(_fake_line())
    assert "\n" not in text
    assert len(text) < 2048
    got = json.loads(text)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches", "metric_parts"):
        assert key in got, key
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in got["roofline"], key
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in got["e2e"], key
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in got["cpu_baseline"], key
    assert got["config"]["T_decision"] == "697/1000" and got["config"]["T_truth"] == "7/10"
    assert abs(got["roofline"]["frac"] - 7171.12 / 6777.0) < 1e-4
    assert got["metric_parts"]["at_equal_recall"] is True
    assert abs(got["value"] - 2.81235e13) / 2.8e13 < 1e-5


def test_headline_drops_optional_keys_before_growing_past_2kb():
    import json
    line = _fake_line()
    line["cpu_baseline"]["sample"] = "x" * 3000
    text = bench.headline_json(line)
    assert len(text) <= 2048
    got = json.loads(text)
    assert "metric_parts" not in got and "sample" not in got["cpu_baseline"]
    assert got["value"] > 0 and "e2e" in got and "roofline" in got


def test_details_go_to_stderr_and_the_headline_is_the_only_stdout_line(capsys, tmp_path):
    import json
    path = tmp_path / "d" / "details.json"
    bench.emit(_fake_line(), {"sweeps": list(range(5000))}, str(path))
    out, err = capsys.readouterr()
    lines = out.strip().splitlines()
    assert len(lines) == 1 and len(lines[0]) < 2048
    assert json.loads(lines[0])["metric"] == bench.METRIC
    assert err.startswith("details: ")
    assert json.loads(path.read_text())["sweeps"][-1] == 4999
