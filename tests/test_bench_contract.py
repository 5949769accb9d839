"""The benchmark's reference arm (the FP64 reference row-sharded over the
host cores) needs no GPU: it must print one JSON line with the keys and types
of the benchmark contract.  The benchmark's own accuracy helpers are checked
against the reference's definitions."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key, typ in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                     ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                     ("dtype", str), ("data", str), ("config", dict), ("impl", str), ("cpu_baseline", dict),
                     ("e2e", dict)):
        assert isinstance(d[key], typ), key
    assert d["impl"] == "reference" and d["metric"] == "hap_message_updates_per_s" and d["value"] > 0
    assert d["vs_baseline"] is None and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "c2"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["sample"] and cb["cpu_model"]
    assert cb["cores"] == len(os.sched_getaffinity(0))
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_benchmark_ari_matches_reference_definition():
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    from oracle import hap_oracle as H

    rng = np.random.default_rng(5)
    for n, ka, kb in ((200, 5, 7), (1000, 40, 3), (500, 500, 500)):
        a, b = rng.integers(0, ka, n) * 7 + 3, rng.integers(0, kb, n)
        assert abs(bench.ari(a, b) - H.adjusted_rand_index(a, b)) <= 1e-12
    same = rng.permutation(300)
    assert bench.ari(same, same) == 1.0
    assert bench.exemplar_counts([[0, 0, 2], [1, 1, 1]]) == [2, 1]
