"""The benchmark's host side without a GPU: the reference arm's JSON line
(the oracle timed on a row sample of the four-class set), the whole-job
throughput arithmetic, and the DRAM-traffic record that is only reported
while the kernel sources it was measured on are unchanged."""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GB/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["n_gpus"] == 1 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench.WORKLOAD and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_job_throughput_counts_every_replica():
    # 1 GB per replica per step, 10 steps, 4 replicas, 2 s for the slowest: 20 GB/s
    assert bench._job_gbs(10**9, 10, 4, 2000.0) == pytest.approx(20.0)


def test_traffic_record_needs_unchanged_sources(tmp_path, monkeypatch):
    import hashlib
    src = tmp_path / "pkg" / "kernel.cu"
    os.makedirs(src.parent)
    src.write_text("__global__ void k() {}\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    os.makedirs(tmp_path / "profiles")
    rec = {"sliced@some_matrix": {"dram_bytes": 123456, "sources": {"pkg/kernel.cu": digest}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("sliced", "some_matrix") == 123456
    assert bench._traffic("no_such_variant", "some_matrix") is None
    with open(src, "a") as f:
        f.write("// changed\n")
    assert bench._traffic("sliced", "some_matrix") is None


def test_committed_traffic_records_are_well_formed():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, r in rec.items():
        if "@" not in key:
            continue
        assert r["dram_bytes"] > 0 and r["sources"]
        for path in r["sources"]:
            assert os.path.exists(os.path.join(ROOT, path)), path


def test_cpu_row_sample_is_strided_over_the_whole_matrix():
    import numpy as np
    import synth
    A = synth.zipf_rows(5000, 5000, 1.5, 3000, seed=1)
    S = bench._row_sample(A, 4, block=64)
    rp = A.rowptr.numpy().astype(np.int64)
    rows = np.concatenate([np.arange(s, min(s + 64, A.n_rows)) for s in range(0, A.n_rows, 256)])
    assert S.n_rows == len(rows) and S.n_cols == A.n_cols
    assert rows[-1] >= A.n_rows - 256  # reaches the end of the matrix
    srp = S.rowptr.numpy().astype(np.int64)
    for k in (0, 1, len(rows) // 2, len(rows) - 1):
        r = rows[k]
        assert np.array_equal(S.colind.numpy()[srp[k]:srp[k + 1]], A.colind.numpy()[rp[r]:rp[r + 1]])
        assert np.array_equal(S.val.numpy()[srp[k]:srp[k + 1]], A.val.numpy()[rp[r]:rp[r + 1]])
    assert srp[-1] == S.nnz == sum(rp[r + 1] - rp[r] for r in rows)
