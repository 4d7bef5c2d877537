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
    bench = _bench()
    vals = {}
    with open(bench.TRAFFIC_SUMMARY) as f:
        for line in f:
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    assert len(vals["k_push.cu sha256"]) == 64
    assert 60.0 < float(vals["dram bytes per particle"]) < 80.0   # 64.5 B algorithmic
    assert 5.0 < float(vals["shared wavefronts per particle"]) < 40.0
    assert float(vals["shared wavefronts per particle"]) < float(vals["l1 data-pipe wavefronts per particle"]) < 40.0
    assert 100.0 < float(vals["fp32 operations per particle"]) < 3000.0


def test_profile_is_used_only_for_the_kernel_it_was_taken_on(tmp_path, monkeypatch):
    bench = _bench()
    src = tmp_path / "k_push.cu"
    src.write_bytes(b"// a kernel\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    md = tmp_path / "profile.md"
    md.write_text(f"- k_push.cu sha256: `{sha}`\n- dram bytes per particle: `64.5`\n"
                  f"- shared wavefronts per particle: `17.0`\n- fp32 operations per particle: `670`\n")
    monkeypatch.setattr(bench, "PUSH_KERNEL_SRC", str(src))
    monkeypatch.setattr(bench, "TRAFFIC_SUMMARY", str(md))
    assert bench.push_profile() == {"tpp": 64.5, "wpp": 17.0, "fpp": 670.0, "wkind": "smem"}
    # the L1 data-pipe count, when present, is the one the binding roofline uses
    md.write_text(md.read_text() + "- l1 data-pipe wavefronts per particle: `18.0`\n")
    assert bench.push_profile() == {"tpp": 64.5, "wpp": 18.0, "fpp": 670.0, "wkind": "l1"}
    src.write_bytes(b"// a changed kernel\n")
    assert bench.push_profile() == {"tpp": None, "wpp": None, "fpp": None, "wkind": None}


def test_missing_profile_gives_nones(tmp_path, monkeypatch):
    bench = _bench()
    monkeypatch.setattr(bench, "TRAFFIC_SUMMARY", str(tmp_path / "absent.md"))
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
