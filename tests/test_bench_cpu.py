"""The benchmark's reference arm (the oracle on the host cores) runs without a GPU and prints
the one JSON line of the contract."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["unit"] == "atom-steps/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_roofline_fraction_on_both_byte_bases():
    """The roofline fields are algorithmic bytes per launch over the launch time, against the
    peak: checked on round numbers (1 GB in 1 ms is 1000 GB/s), for the half-matrix basis and
    the stored-bytes basis reported beside it."""
    b = _bench()
    stages = {"qeq": {"ms_per_step": 1.0}}
    costs = {"qeq": {"bytes": 1.0e9, "spmv": 8}, "qeq_full_storage": {"bytes": 2.0e9, "spmv": 8}}
    r = b.roofline("qeq", stages, costs, {"hbm_gbs": 4000.0, "source": "measured"}, 4)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak_source"] == "measured"
    assert abs(r["achieved"] - 1000.0) < 1e-9 and abs(r["frac"] - 0.25) < 1e-12
    assert r["launch_ms"] == 1.0 and r["algorithmic_bytes_per_launch"] == 1.0e9
    assert abs(r["full_storage_basis"]["achieved"] - 2000.0) < 1e-9
    assert abs(r["full_storage_basis"]["frac"] - 0.5) < 1e-12
    # a stage without a byte model is reported as ALU-bound with no fraction
    r2 = b.roofline("angles", {"angles": {"ms_per_step": 0.07}}, costs, {"hbm_gbs": 4000.0, "source": "m"}, 4)
    assert r2["bound"] == "alu" and r2["frac"] is None


def test_qeq_traffic_follows_the_profiled_source(tmp_path, monkeypatch):
    """roofline.traffic uses the committed ncu summary only while qeq.cu is the file those
    counters were taken from: the summary names its SHA-256, and a changed source gives None."""
    import hashlib
    b = _bench()
    src = open(os.path.join(ROOT, "paper_1706_07772_gb300", "csrc", "qeq.cu"), "rb").read()
    (tmp_path / "paper_1706_07772_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_1706_07772_gb300" / "csrc" / "qeq.cu").write_bytes(src)
    summary = "traffic_bytes_per_spmv: 123456\nsource_sha256 qeq.cu: %s\n" % hashlib.sha256(src).hexdigest()
    (tmp_path / "profiles" / "k_cg_petn32k_mixed.md").write_text(summary)
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.cg_traffic_per_spmv() == 123456
    (tmp_path / "paper_1706_07772_gb300" / "csrc" / "qeq.cu").write_bytes(src + b"\n// edited\n")
    assert b.cg_traffic_per_spmv() is None
    (tmp_path / "profiles" / "k_cg_petn32k_mixed.md").write_text("no figures here\n")
    assert b.cg_traffic_per_spmv() is None

