"""The reference arm of bench.py (the FP64 oracle timed on the host cores)
keeps the one-JSON-line contract, on the CPU: same metric, unit and config
keys as the GPU arm, `impl` = reference, a cpu_baseline describing the run
and an e2e object with zero copied bytes; under a multi-rank launch only
rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    out = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in out, k
    assert out["impl"] == "reference"
    assert out["steps"] == 1 and out["warmup"] == 3          # at least 3 warm-up steps
    assert out["value"] > 0 and out["higher_is_better"] is True
    assert out["config"]["workload"].startswith("cavity_cube")
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # the measured work: DOF x steps / time
    assert abs(out["value"] * out["ms_per_step"] * 1e-3 - out["config"]["dof"]) < 1e-6 * out["config"]["dof"]


def test_reference_arm_other_ranks_exit_quietly():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_measured_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    # roofline.traffic comes from profiles/force_traffic.txt only while its
    # sources_sha matches the kernel sources; otherwise null
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    h = b.kernel_sources_hash()
    p = tmp_path / "traffic.txt"
    p.write_text("# comment\nsources_sha %s\nmixed_walsh_gen_tc_pair 81.0e6\n" % h)
    monkeypatch.setattr(b, "TRAFFIC_FILE", str(p))
    assert b.measured_traffic("mixed_walsh_gen_tc_pair") == 81.0e6
    assert b.measured_traffic("mixed_tensor_gen_simt_pair") is None
    p.write_text("sources_sha 0000000000000000\nmixed_walsh_gen_tc_pair 81.0e6\n")
    assert b.measured_traffic("mixed_walsh_gen_tc_pair") is None
    monkeypatch.setattr(b, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert b.measured_traffic("mixed_walsh_gen_tc_pair") is None
