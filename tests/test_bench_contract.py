"""CPU tests of bench.py's reference arm (the FP64 oracle timed on the host cores): the JSON line
it prints carries every key of the benchmark contract, and under a multi-rank launch only rank 0
works and prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return p


def test_reference_line_has_the_contract_keys():
    p = _run()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 0)
    assert abs(d["ms_per_step"] - 1000.0 / d["value"]) <= 1e-6 * d["ms_per_step"]
    assert d["vs_baseline"] is None and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    # one step is one full steady solve of the workload, timed (not extrapolated)
    assert len(cb["per_solve_s"]) == 1 and abs(cb["per_solve_s"][0] - d["ms_per_step"] / 1000.0) < 1.0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [ln for ln in p.stdout.splitlines() if ln.strip().startswith("{")]


def test_unet_layer_table_sums_to_the_network_flops():
    """The per-convolution accounting of the U-Net report adds up to the FLOPs the TFLOP/s
    figures divide by (2 k^2 C_in C_out per output pixel), at any batch."""
    import bench
    for B in (1, 16):
        rows = bench.unet_layer_table(256, B)
        assert [r["layer"] for r in rows][:2] == ["e0a", "e0b"] and rows[-1]["layer"] == "head"
        assert abs(sum(r["gflop"] for r in rows) * 1e9 - bench.unet_conv_flops() * B) <= 1e-6 * bench.unet_conv_flops() * B
        assert all(r["activation_mb"] > 0 and r["weight_kb"] > 0 for r in rows)
