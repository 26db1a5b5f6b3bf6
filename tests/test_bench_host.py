"""Host-side logic of bench.py: the algorithmic bytes model, the BFS and relabel rates,
the measured peak and the recorded-traffic guard (no GPU needed)."""
import json
import os

import pytest

import bench   # noqa: E402  (the repository root is on sys.path, see conftest.py)


def _profile(**kw):
    P = dict(n=1000, nnz=8000, queue=1, nrounds=4, queue_clusters=3, scan_listed=100, scan_rows=80,
             scan_arcs=640, bfs_visited=3_000_000, bfs_arcs=24_000_000, corridor_n=250, corridor_arcs=2000,
             relabels=5, gr_arcs=10_000_000,
             phase_ms=dict(bfs=2.0, select=0, lid=0, build=0, flow=0, relabel=0.0, ret=0),
             cluster_phase_ms=dict(load=0, flow=0, ret=0, reach=0, scc=0, members=0, relabel=4.0))
    P["phase_ms"]["return"] = 0
    P["cluster_phase_ms"]["return"] = 0
    P.update(kw)
    return P


def test_bytes_model_counts_each_phase():
    P = _profile()
    bm = bench.bytes_model(P)
    assert bm["scan"] == 8 * 100 + 8 * 80 + 8 * 640
    assert bm["bfs"] == 16 * 3_000_000 + 12 * 24_000_000
    assert bm["build"] == 12 * 250 + 28 * 2000
    assert bm["cluster"] == 52 * 250 + 28 * 2000
    # the queue sweep: every phase in one kernel, ids from the visit list alone
    assert bm["queue"] == bm["scan"] + bm["step"] + bm["cluster"]
    round_by_round = bench.bytes_model(dict(P, queue=0))
    assert round_by_round["step"] - bm["step"] == (1000 // 8) * 4


def test_phase_rates_of_a_cluster_and_a_grid_relabel():
    P = _profile()
    r = bench.phase_rates_of(P, 1000.0, npairs=7)
    bfs_bytes = 16 * 3_000_000 + 12 * 24_000_000
    assert r["bfs"]["bytes"] == bfs_bytes
    assert r["bfs"]["gbs"] == pytest.approx(bfs_bytes / 2e-3 / 1e9, abs=0.05)
    assert r["bfs"]["frac"] == pytest.approx(bfs_bytes / 2e-3 / 1e9 / 1000.0, abs=1e-4)
    assert r["relabel"]["arcs_per_s"] == pytest.approx(10_000_000 / 4e-3, rel=1e-6)
    assert "shared memory" in r["relabel"]["memory"] and "gbs" not in r["relabel"]
    assert r["schedule"] == "queue" and r["clusters"] == 3 and r["pairs"] == 7
    # the grid-wide relabel reads head, reverse residual and label per arc from HBM
    g = bench.phase_rates_of(_profile(queue=0, phase_ms=dict(P["phase_ms"], relabel=8.0),
                                      cluster_phase_ms=dict(P["cluster_phase_ms"], relabel=0.0)), 1000.0, 1)
    assert g["relabel"]["memory"] == "hbm"
    assert g["relabel"]["gbs"] == pytest.approx(12 * 10_000_000 / 8e-3 / 1e9, abs=0.05)


def test_recorded_traffic_is_used_only_for_the_current_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(
        {"queue_kernel": {"source_hash": "abc", "dram_bytes_per_launch_full": 123}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.recorded_traffic("queue_kernel")[0] == 123
    assert bench.recorded_traffic("cluster_flow_kernel") == (None, None)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "def")   # the kernels changed since
    assert bench.recorded_traffic("queue_kernel") == (None, None)


def test_measured_peak_reads_the_measured_copy_rate():
    peak, kind = bench.measured_peak_gbs()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak > 1000
    else:
        assert kind == "fallback"
