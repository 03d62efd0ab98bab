"""bench.py's reference arm on the CPU: the oracle timed on the host cores,
printing one JSON line with the fields the benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--reference-budget-s", "1"],
                       capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Gsamples/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["steps"] == 2 and d["higher_is_better"] is True


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       cwd=ROOT, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_transform_precision_record_on_cpu_tensors():
    """The benchmark's precision record (run on the GPU output in the real
    benchmark) on host tensors holding the oracle's own outputs: uniforms
    report zero mismatching bit patterns, and one planted wrong bit is
    counted; normals rounded from FP64 to FP32 report an error within a
    float's rounding, and the tail statistics count the |z| >= 5 values."""
    import numpy as np
    import torch

    import bench
    import oracle

    key = int(oracle.make_keys(11, 1)[0])
    n = (1 << 16) + 6
    u = oracle.uniform_f32(key, 0, n)
    buf = torch.from_numpy(u.view(np.uint8).copy())
    rec = bench.transform_precision(torch, np, "uniform_f32", buf, key, n, chunk=1 << 14)
    assert rec["mismatching_bit_patterns"] == 0 and rec["outputs"] == n
    buf[4 * 777] ^= 1
    assert bench.transform_precision(torch, np, "uniform_f32", buf, key, n,
                                     chunk=1 << 14)["mismatching_bit_patterns"] == 1
    b16 = oracle.uniform_bf16(key, 0, n)
    rec = bench.transform_precision(torch, np, "uniform_bf16", torch.from_numpy(b16.view(np.uint8).copy()),
                                    key, n, chunk=1 << 14)
    assert rec["mismatching_bit_patterns"] == 0
    z64 = oracle.normal_f64(key, 0, n)
    z32 = z64.astype(np.float32)
    rec = bench.transform_precision(torch, np, "normal_f32", torch.from_numpy(z32.view(np.uint8).copy()),
                                    key, n, chunk=1 << 14)
    assert 0 < rec["max_abs_core"] <= 5 * 2.0 ** -24 * 4
    assert rec["tail_count"] == int(np.count_nonzero(np.abs(z64) >= 5))
    assert rec["max_abs_z"] == float(np.abs(z64).max())


def test_oracle_batch_rate_writes_the_prefix_streams():
    """The per-config oracle timing of the ragged batch splits the first
    streams over threads; it reports a positive rate and a sample naming
    the streams it ran."""
    import numpy as np

    import bench
    from paper_2004_06278_gb300 import workloads

    b = workloads.small_ragged_batch(64, seed=3, max_len=5000, gap_max=0)
    rec = bench.oracle_batch_rate(np, b, prefix=int(b.total // 2))
    assert rec["value"] > 0 and rec["kind"] == "oracle" and rec["cores"] >= 1
    assert "streams" in rec["sample"] and rec["single_thread"]["value"] > 0
