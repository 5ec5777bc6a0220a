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
