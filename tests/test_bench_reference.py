"""bench.py's reference arm (the CPU oracle as it stands, one single-threaded
process per core, each on its own bounded sample of the workload) on a tiny
sample: it needs no GPU and prints one JSON line with the contract's keys --
the metric and unit of the GPU arm, the measured time per step, a config
stating the particles actually stepped, a cpu_baseline describing the run
and an e2e object with no host-device bytes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run(
        [sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
         "--cpu-sample-per-core", "2e4", "--cpu-procs", "2"], cwd=ROOT, capture_output=True,
        text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["unit"] == "particle-steps/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["dtype"] == "f64" and d["data"] == "synthetic"
    cfg = d["config"]
    assert cfg["n_per_species"] == 2 * 20000 and cfg["grid"] == [256, 256]
    assert cfg["sample"]["processes"] == 2 and cfg["sample"]["n_per_species_per_process"] == 20000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"]
    assert "2 single-threaded oracle processes" in cb["sample"] and "257x257" in cb["sample"]
    # ms_per_step is the measured wall time of one step of the sample
    assert abs(cb["particles_per_step"] / (d["ms_per_step"] / 1e3) - d["value"]) <= 1e-6 * d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
