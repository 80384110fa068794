"""The benchmark's accounting helpers, on CPU:

- each kernel's share of a K-step record-path run weights its per-launch time
  by how often it runs (the scatter, the last step and the placement once per
  run, the inner step and fix-up K - 1 times, the others every step), so the
  shares agree with a launch list of the run;
- DRAM traffic and warp instructions from the committed ncu capture are used
  only while the kernel's sources are the ones captured, and are scaled by N;
- the issue rate is the measured instructions per second against four warp
  schedulers per SM at the given clock.
"""
import json

import bench


def test_run_shares_weight_kernels_by_launches_per_run():
    avg = {"k_rec_scatter": 0.5, "k_rec_split": 0.5, "k_rec_scan": 0.02, "k_rec_step": 1.5, "k_rec_fixup": 0.01,
           "k_rec_step_last": 1.3, "k_rec_fixup_last": 0.01, "k_rec_place": 1.3}
    steps = 50
    sh = bench._run_shares(avg, steps)
    total = (0.5 + 1.3 + 0.01 + 1.3) + steps * (0.5 + 0.02) + (steps - 1) * (1.5 + 0.01)
    assert abs(sum(sh.values()) - 1.0) < 1e-12
    assert abs(sh["k_rec_step"] - (steps - 1) * 1.5 / total) < 1e-12
    assert abs(sh["k_rec_split"] - steps * 0.5 / total) < 1e-12
    for once in ("k_rec_scatter", "k_rec_step_last", "k_rec_place"):
        assert abs(sh[once] - avg[once] / total) < 1e-12
    # a path whose kernels all run every step: shares of the per-step times
    sh2 = bench._run_shares({"k_a": 1.0, "k_b": 3.0}, 10)
    assert abs(sh2["k_a"] - 0.25) < 1e-12 and abs(sh2["k_b"] - 0.75) < 1e-12


def test_traffic_and_issue_rate_follow_the_captured_sources(tmp_path, monkeypatch):
    digest = bench._kernel_sources_digest("k_rec_step")
    prof = tmp_path / "profiles"
    prof.mkdir()
    ent = {"dram_bytes_per_launch": 600.0, "warp_inst_per_launch": 1000.0, "n": 100, "sources": digest}
    (prof / "traffic.json").write_text(json.dumps({"wl": {"k_rec_step": ent}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the kernel sources are read from the package, not from ROOT
    monkeypatch.setattr(bench, "_kernel_sources_digest", lambda k="": digest)
    assert bench._traffic_for("wl", "k_rec_step", digest, 400) == 2400.0
    r = bench._issue_rate("wl", "k_rec_step", 2.0, 400, 2000.0, 10)
    assert r["warp_instructions_per_launch"] == 4000.0
    assert abs(r["achieved"] - 4000.0 / 2e-3) < 1e-6
    assert r["peak"] == 4.0 * 10 * 2000e6
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    # another kernel source: no figure
    monkeypatch.setattr(bench, "_kernel_sources_digest", lambda k="": "0" * 16)
    assert bench._traffic_for("wl", "k_rec_step", digest, 400) is None
    assert bench._issue_rate("wl", "k_rec_step", 2.0, 400, 2000.0, 10) is None
