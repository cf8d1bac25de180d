"""bench.py's reference arm (the CPU oracle on every host core) on CPU: one
JSON line with the keys the benchmark contract names, on the same metric,
unit and workload as the GPU arm, a refusal to run the batch workload's
~35 GB of tables, and the oracle's time to the final ln f."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_line():
    import bench
    from paper_1508_02748_gb300 import workloads
    d = _run("--impl", "reference", "--steps", "2", "--warmup", "3")
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "trials/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "rewl_L32_16x4_w32"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    cores = bench.host_cores()
    assert cb["kind"] == "oracle" and cb["cores"] == cores and cb["value"] == d["value"] and cb["sample"]
    assert cb["cpu_model"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # 2 cycles x 10^4 trials x (64 windows x the sample's walkers) in each process, in the slowest one's time
    wpw = bench.oracle_sample_walkers(workloads.REWL_L32)
    assert wpw == 2
    trials = cores * 2 * 10_000 * 64 * wpw
    assert abs(d["value"] * d["ms_per_step"] * 2 / 1e3 - trials) < 1e-3 * trials


def test_reference_arm_warmup_floor():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert d["warmup"] >= 3


def test_reference_arm_refuses_batch():
    d = _run("--impl", "reference", "--workload", "batch_24_mixed_L16_24_32_48", "--steps", "1")
    assert d["impl"] == "reference" and "unavailable" in d


def test_reference_time_to_serial_L4():
    """The oracle run to its final ln f, seed by seed: the serial L = 4 walker
    (one window, one walker) meets the enumerated g(E) to a few percent, and a
    seed gives the same run twice."""
    d = _run("--impl", "reference", "--time-to", "--workload", "serial_wl_L4", "--replicates", "2")
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert [r["seed"] for r in d["runs"]] == [20151811, 20151812]
    for r in d["runs"]:
        assert not r["capped"] and r["iterations"] == 21
        assert 0 < r["mean_eps_E_marginal_vs_exact"] < 0.026
    again = _run("--impl", "reference", "--time-to", "--workload", "serial_wl_L4", "--replicate", "1")
    assert again["runs"][0]["cycles"] == d["runs"][1]["cycles"]
    assert again["runs"][0]["mean_eps_E_marginal_vs_exact"] == d["runs"][1]["mean_eps_E_marginal_vs_exact"]
