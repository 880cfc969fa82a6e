"""The benchmark's reference arm (the oracle on the host) keeps the one-JSON-line contract."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, env=None):
    e = dict(os.environ, **(env or {}))
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         env=e, cwd=ROOT, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    return [json.loads(line) for line in out.stdout.splitlines() if line.startswith("{")]


def test_reference_arm_prints_one_line_with_the_contract_keys():
    lines = _run("--impl", "reference", "--workload", "uniform_100x3_1e4", "--steps", "2", "--warmup", "1")
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == "CD-sweep nnz-updates/s"
    assert d["unit"] == "entry-mode updates/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "uniform_100x3_1e4"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_on_other_ranks_and_other_workloads():
    assert _run("--impl", "reference", "--workload", "uniform_100x3_1e4", "--steps", "1", "--warmup", "1",
                env={"RANK": "1", "WORLD_SIZE": "2"}) == []
    lines = _run("--impl", "reference", "--workload", "batch_256_jobs", "--steps", "1", "--warmup", "1")
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and "unavailable" in lines[0]


def _copy_tree_for_traffic(tmp_path):
    """The files profiled_traffic reads: the committed summaries and the kernel sources."""
    import shutil
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "profiles"), root / "profiles")
    shutil.copytree(os.path.join(ROOT, "paper_1904_02603_gb300", "csrc"), root / "paper_1904_02603_gb300" / "csrc")
    return root


def test_roofline_traffic_comes_from_the_summary_while_its_sources_match(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    root = _copy_tree_for_traffic(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    text = (root / "profiles" / "sweep_task_tc_kernel_zipf_1e5x3_1e7.md").read_text()
    want = float(next(l for l in text.splitlines() if l.startswith("dram_bytes_per_launch:")).split(":", 1)[1])
    traffic, source = bench.profiled_traffic("zipf_1e5x3_1e7", True)
    assert traffic == want and "sweep_task_tc_kernel_zipf_1e5x3_1e7.md" in source
    # a workload without a summary, and a kernel source changed after the capture: no traffic
    assert bench.profiled_traffic("uniform_1e4x4_5e7", True)[0] is None
    src = root / "paper_1904_02603_gb300" / "csrc" / "tc_delta.cuh"
    src.write_text(src.read_text() + "\n// edited after the capture\n")
    traffic, why = bench.profiled_traffic("zipf_1e5x3_1e7", True)
    assert traffic is None and "changed" in why
