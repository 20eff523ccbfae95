"""Host logic of bench.py (no GPU): the measured DRAM traffic of a kernel counts
only while the kernel's sources are the ones it was captured on, every bench
workload is named with a kernel family whose sources exist, and the JSON
contract's fixed keys are produced by the reference arm's line."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_needs_the_captured_sources(tmp_path, monkeypatch):
    kernel = "stage2d_kernel 16x16 fp32 mhd, stage 2"
    entry = {"dram_bytes_per_launch": 123, "src_sha": bench._src_sha(kernel), "captured": "t"}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps({"w": {kernel: entry}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash is of the package sources, which stay where they are
    monkeypatch.setattr(bench, "_src_sha", lambda k: entry["src_sha"] if k == kernel else "x")
    assert bench._traffic(kernel, "w") == 123
    assert bench._traffic(kernel, "other workload") is None
    monkeypatch.setattr(bench, "_src_sha", lambda k: "changed")
    assert bench._traffic(kernel, "w") is None


def test_source_hash_covers_the_family_and_shared_headers():
    csrc = os.path.join(ROOT, "paper_1305_5536_gb300", "csrc")
    for fam, files in bench._FAMILY_SOURCES.items():
        for f in files + ("dg_physics.cuh", "dg_common.cuh", "dg_weno.cuh"):
            assert os.path.exists(os.path.join(csrc, f)), (fam, f)
        h = bench._src_sha(fam + " 8x8 fp32")
        assert len(h) == 16 and h != bench._src_sha("unknown_kernel")


def test_every_workload_is_described_and_restarts_within_its_safe_range():
    for name, w in bench.WORKLOADS.items():
        assert w["desc"] and w["eq"] in ("euler", "mhd") and w["dim"] in (2, 3), name
        assert 0 < w.get("restart", bench.RESTART_STEPS) <= bench.RESTART_STEPS, name
        m = bench._metric(w)
        assert ("MUSCL-Hancock" in m) == (w.get("integrator") == "mh"), name


def test_reference_arm_line_keeps_the_contract(capsys, monkeypatch):
    """`bench.py --impl reference` on the small 64^2 workload: one JSON line with
    the contract's keys, the oracle described as the CPU baseline, and an e2e
    entry without device copies."""
    import argparse
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    args = argparse.Namespace(workload="smooth_wave_64", steps=2, warmup=1, gpus=1,
                              impl="reference", no_cpu_baseline=False, no_adjoint=True)
    bench.run_reference(args)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["metric"] == bench._metric(bench.WORKLOADS["smooth_wave_64"])
