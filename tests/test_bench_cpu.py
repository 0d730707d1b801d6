"""The benchmark's reference arm (the CPU oracle timed on the host cores)
keeps the JSON-line contract, on a small graph, with no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--scale", "12", "--edges-log2", "15", "--steps", "2", "--warmup", "1"]


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"] + SMALL,
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [line for line in out.stdout.splitlines() if line.strip()]


def test_reference_arm_prints_one_contract_line():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "rmat12_e15"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_ncu_traffic_only_for_its_launch_shape_and_sources(monkeypatch):
    """roofline.traffic is an ncu figure of one launch shape of one kernel
    build: another shape, or sources that no longer match the digest taken
    with the capture, report null."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.NCU_TRAFFIC, "no traffic figures recorded"
    (fam, workload, words, group), (nbytes, srcs, digest) = next(iter(bench.NCU_TRAFFIC.items()))
    monkeypatch.setattr(bench, "_src_digest", lambda paths: digest)
    assert bench.traffic_bytes(fam, workload, (words, group)) == nbytes
    assert bench.traffic_bytes(fam, workload, (words, 2 * group)) is None
    assert bench.traffic_bytes(fam, "another_workload", (words, group)) is None
    monkeypatch.setattr(bench, "_src_digest", lambda paths: "0" * 64)
    assert bench.traffic_bytes(fam, workload, (words, group)) is None


def test_source_digest_ignores_comments_and_layout(tmp_path, monkeypatch):
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_under_test2", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    a.write_text("int f(int x) { return x + 1; }  // add one\n")
    b.write_text("/* add one */\nint f(int x)\n{\n    return x + 1;\n}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._src_digest(("a.cu",)) == bench._src_digest(("b.cu",))
    b.write_text("int f(int x) { return x + 2; }\n")
    assert bench._src_digest(("a.cu",)) != bench._src_digest(("b.cu",))
