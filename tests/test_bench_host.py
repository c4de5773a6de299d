"""Host logic of bench.py (no GPU): the reference arm's JSON line, the ncu
traffic lookup keyed by the leaf-kernel source, peak lookup and the clock
sampler without nvidia-smi."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def bench():
    # imported here, not at collection: bench.py sets process-wide CUDA
    # environment defaults when it is imported
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_reference_arm_line(bench):
    # a 127^2 sample keeps this CPU test short (the default is the 1023^2 workload itself)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--ref-sample-n", "128"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_oracle_sample_all_cores(bench):
    """The all-cores leg forks workers after the setup and reports their
    aggregate rate (small sample: 127^2, one step each, two workers)."""
    r = bench.run_oracle_subprocess(128, 1, 0, 1e-6, procs=2)
    assert r["steps"] == 1 and r["steps_per_s_sample"] > 0 and r["iters_per_step"] >= 1
    ac = r["all_cores"]
    assert ac["procs"] == 2 and ac["steps_per_s_sample"] > 0 and ac["iters_per_step"] >= 1


def test_traffic_follows_leaf_source(bench, tmp_path, monkeypatch):
    h = bench.leaf_kernel_source_hash()
    assert len(h) == 64 and h == bench.leaf_kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    doc = {"leaf_kernel_sha256": h,
           "kernels": {"cell_bwd_l0": {"dram_bytes_per_launch_full": 123456789}}}
    (prof / "traffic.json").write_text(json.dumps(doc))
    # the lookup reads profiles/ under ROOT and hashes the sources under ROOT
    csrc = tmp_path / "paper_2004_05566_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("apply.cu", "internal.h"):
        src = os.path.join(ROOT, "paper_2004_05566_gb300", "csrc", f)
        (csrc / f).write_text(open(src).read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("cell_bwd_l0") == 123456789.0
    assert bench.kernel_traffic("cell_fwd_l0") is None
    # a change inside the leaf-kernel section invalidates the figures
    a = (csrc / "apply.cu").read_text()
    marker = "// ------------------------------------------------------------ TMA-staged cells"
    (csrc / "apply.cu").write_text(a.replace(marker, marker + "\n// edited"))
    assert bench.kernel_traffic("cell_bwd_l0") is None


def test_find_peak_nested(bench):
    d = {"gpu": {"hbm": {"hbm_gbs": 6793.1}, "bf16_tflops": 1800.0}}
    assert bench._find_peak(d, ("hbm_gbs",)) == 6793.1
    assert bench._find_peak(d, ("nothing",)) is None


def test_clock_sampler_without_nvidia_smi(bench, tmp_path, monkeypatch):
    monkeypatch.setenv("HIFCN_CLOCKS_DIR", str(tmp_path))
    monkeypatch.setenv("PATH", str(tmp_path))  # no nvidia-smi on PATH
    c = bench.ClockSampler(0)
    assert c.path.startswith(str(tmp_path))
    c.start()
    r = c.stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]


def test_oracle_only_in_the_baseline_leg():
    """bench.py imports the oracle only inside the CPU sample (the baseline and
    reference legs, run in their own process); the timed GPU arm never does."""
    import ast
    src = open(os.path.join(ROOT, "bench.py")).read()
    tree = ast.parse(src)
    hosts = []
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == "oracle":
                    hosts.append(fn.name)
                if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle"
                                                        for a in node.names):
                    hosts.append(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))
           and "oracle" in ast.dump(n)]
    assert not top
    assert set(hosts) == {"oracle_sample"}, hosts
