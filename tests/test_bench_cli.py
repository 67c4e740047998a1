"""bench.py's reference arm (the FP64 oracle on the host cores) prints the
contract's JSON line; CPU only, on a tiny sample."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload", ["beam2d_64", "walker2d_128", "walker3d_128"])
def test_reference_arm_json_line(orc, workload):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", workload, "--cpu-sample-steps", "2"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["value"] > 0 and out["higher_is_better"] is True
    assert out["config"]["workload"].startswith(workload)
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["unit"] == out["unit"]


def test_recorded_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    """roofline.traffic comes from profiles/traffic.json only while the
    particle kernels' sources hash to the value recorded with the capture."""
    sys.path.insert(0, ROOT)
    import bench

    cls = "forward particle (G2P+P2G)"
    rec = {"walker2d_128": {cls: {"kernel": "k", "dram_bytes_per_launch": 1234, "profile": "p.md",
                                  "kernel_sources_sha256_16": bench.kernel_source_hash()}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    csrc = tmp_path / "paper_2503_22767_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        (csrc / name).write_bytes(open(os.path.join(ROOT, "paper_2503_22767_gb300", "csrc", name), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("walker2d_128", cls) == (1234.0, "p.md")
    # another workload or kernel class: nothing recorded
    assert bench.recorded_traffic("walker2d_128", "grid operation")[0] is None
    assert bench.recorded_traffic("plate3d_64", cls)[0] is None
    # a kernel source changes: the recorded figure no longer applies
    with open(csrc / bench.KERNEL_SOURCES[0], "ab") as fh:
        fh.write(b"\n// changed\n")
    value, why = bench.recorded_traffic("walker2d_128", cls)
    assert value is None and "changed" in why


def test_committed_traffic_records_are_well_formed():
    """Every committed traffic figure names its kernel, a positive byte count,
    an existing profile summary and the source hash it was taken on."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for workload, classes in rec.items():
        if workload.startswith("_"):
            continue
        for cls, e in classes.items():
            assert e["kernel"].startswith("k_") and e["dram_bytes_per_launch"] > 0, (workload, cls)
            assert len(e["kernel_sources_sha256_16"]) == 16
            assert os.path.exists(os.path.join(ROOT, e["profile"])), e["profile"]
