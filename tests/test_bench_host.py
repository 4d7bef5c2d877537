"""Host logic of bench.py (no GPU): the committed push-kernel profile is
read only while the kernel source still has the hash it was taken on, and
its per-particle figures parse; the reference arm (the FP64 oracle on the
host) prints the contract's JSON line."""
import argparse
import hashlib
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    import sys

    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench

    return bench


def test_committed_profile_has_every_figure():
    import json

    bench = _bench()
    with open(bench.TRAFFIC_SUMMARY) as f:
        vals = json.load(f)
    assert len(vals["kernel_source_sha256"]) == 64
    assert 60.0 < float(vals["dram_bytes_per_particle"]) < 80.0   # 64.5 B algorithmic
    assert 5.0 < float(vals["shared_wavefronts_per_particle"]) < 40.0
    assert float(vals["shared_wavefronts_per_particle"]) < float(vals["l1_wavefronts_per_particle"]) < 40.0
    assert 100.0 < float(vals["fp32_ops_per_particle"]) < 3000.0
    assert "ncu" in vals["command"] and "--clock-control none" in vals["command"]


def test_profile_is_used_only_for_the_kernel_it_was_taken_on(tmp_path, monkeypatch):
    import json

    bench = _bench()
    src = tmp_path / "k_push.cu"
    src.write_bytes(b"// a kernel\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    js = tmp_path / "profile.json"
    fig = {"kernel_source_sha256": sha, "dram_bytes_per_particle": 64.5, "shared_wavefronts_per_particle": 17.0,
           "fp32_ops_per_particle": 670}
    js.write_text(json.dumps(fig))
    monkeypatch.setattr(bench, "PUSH_KERNEL_SRC", str(src))
    monkeypatch.setattr(bench, "TRAFFIC_SUMMARY", str(js))
    assert bench.push_profile() == {"tpp": 64.5, "wpp": 17.0, "fpp": 670.0, "wkind": "smem"}
    # the L1 data-pipe count, when present, is the one the binding roofline uses
    js.write_text(json.dumps(dict(fig, l1_wavefronts_per_particle=18.0)))
    assert bench.push_profile() == {"tpp": 64.5, "wpp": 18.0, "fpp": 670.0, "wkind": "l1"}
    src.write_bytes(b"// a changed kernel\n")
    assert bench.push_profile() == {"tpp": None, "wpp": None, "fpp": None, "wkind": None}


def test_missing_profile_gives_nones(tmp_path, monkeypatch):
    bench = _bench()
    monkeypatch.setattr(bench, "TRAFFIC_SUMMARY", str(tmp_path / "absent.json"))
    assert bench.push_profile() == {"tpp": None, "wpp": None, "fpp": None, "wkind": None}


@pytest.mark.parametrize("shape", ["tsc", "cic", "pcs"])
def test_shape_table(shape):
    bench = _bench()
    assert bench.SHAPE[shape] in (1, 2, 3)


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference runs the oracle on the host and prints one
    JSON line with the measured arm's metric, unit and config.workload."""
    import json
    import subprocess
    import sys

    bench = _bench()
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0
    args = argparse.Namespace(shape="tsc", gather="momentum")
    assert d["config"]["workload"] == bench.thermal_workload_name(args, 256)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
