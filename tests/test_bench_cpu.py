"""The benchmark's reference arm on the CPU: `bench.py --impl reference`
times the oracle on the host cores and prints one JSON line of the
contract's form on the same workload as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--cpu-seconds", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == "cell-updates/s" and d["unit"] == "cell-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"] == bench.BATCHED_WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_profiled_traffic_only_for_the_kernel_it_was_taken_on(tmp_path, monkeypatch):
    """`roofline.traffic` comes from a committed ncu summary only while the
    kernel's sources hash to the value the summary records; a stale or
    missing summary gives null, never another kernel's bytes."""
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    prof = tmp_path / "summary.md"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.PROFILES, "resident", (str(prof), ["kernel.cu"]))
    assert bench.profiled_traffic("resident") is None  # no summary
    h = bench.kernel_source_hash("resident")
    prof.write_text(f"# k\n\ntraffic_bytes_per_launch: 123456\nkernel_source_sha256: {h}\n")
    assert bench.profiled_traffic("resident") == 123456
    src.write_text("__global__ void k() { }\n")  # the kernel changed since the capture
    assert bench.profiled_traffic("resident") is None


def test_committed_summaries_carry_traffic_and_a_source_hash():
    """Every summary the bench reads names its DRAM bytes per launch and the
    hash of the sources it was taken on."""
    sys.path.insert(0, ROOT)
    import bench
    for kind, (path, files) in bench.PROFILES.items():
        text = open(path).read()
        fields = dict(ln.split(":", 1) for ln in text.splitlines()
                      if ln.startswith(("traffic_bytes_per_launch:", "kernel_source_sha256:")))
        assert int(fields["traffic_bytes_per_launch"]) > 0, kind
        assert len(fields["kernel_source_sha256"].strip()) == 64, kind
        assert all(os.path.exists(os.path.join(ROOT, f)) for f in files), kind
