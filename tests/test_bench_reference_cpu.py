"""bench.py on the CPU: its reference arm (the FP64 oracle on the host
cores) prints one JSON line with the contract's keys on rank 0 and nothing on
the other ranks of a multi-rank launch; the hash that ties the committed ncu
figures to the kernel's sources."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env):
    env = dict(os.environ, **extra_env)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_prints_the_contract_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["dtype"] == "f64" and d["unit"] == "evals/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_do_no_work():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_capture_hash_covers_the_kernel_and_its_launcher_only(tmp_path, monkeypatch):
    """The committed ncu figures stay valid while the kernel's function, its
    launcher and the device header are unchanged: an edit elsewhere in the
    file keeps the hash, an edit inside the kernel changes it."""
    sys.path.insert(0, ROOT)
    import bench
    src = open(os.path.join(ROOT, "paper_2012_08221_gb300", "csrc", "fwd.cu")).read()
    body = bench.kernel_source("paper_2012_08221_gb300/csrc/fwd.cu", "k_xfxq2")
    assert body.startswith("template <") and "k_xfxq2(" in body and body.endswith("}")
    assert "k_xfxq2_pw" not in body
    d = tmp_path / "paper_2012_08221_gb300" / "csrc"
    d.mkdir(parents=True)
    files = ["paper_2012_08221_gb300/csrc/fwd.cu::k_xfxq2", "paper_2012_08221_gb300/csrc/fwd.cu::launch_matrix"]
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (d / "fwd.cu").write_text(src)
    h0 = bench.source_hash(files)
    (d / "fwd.cu").write_text(src + "\n// a comment outside the kernel\n")
    assert bench.source_hash(files) == h0
    (d / "fwd.cu").write_text(src.replace("if (lane == 0) bulk_wait_all();", "if (lane == 0)  bulk_wait_all();"))
    assert bench.source_hash(files) != h0
