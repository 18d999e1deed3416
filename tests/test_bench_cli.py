"""bench.py on the CPU: every default extra row has its function, the traffic
figure is read from a committed profile only while the kernel's sources are
unchanged, and the reference arm (the oracle on the host) prints one valid
JSON line."""
import json
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))


def test_default_rows_have_functions():
    import bench
    for name in ("extra_rows", "slope_split_row", "d8_4096_row", "long_rivers_row", "batch_rows",
                 "adjoint_row", "richardson_row", "fill_row", "d8_crop_check", "run_reference",
                 "profile_traffic", "count_launches"):
        assert callable(getattr(bench, name)), name
    defaults = bench.parse.__code__.co_consts
    rows = [c for c in defaults if isinstance(c, str) and "slope_split" in c]
    assert rows, "default --rows lists the slope-split sibling"


def test_profile_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    csrc = tmp_path / "paper_2606_12800_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES["k_local_d8"]:
        (csrc / name).write_text("// " + name + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.sources_sha("k_local_d8")
    (prof / "k.md").write_text("traffic-record: kernel=k_local_d8 cells=100 dram_bytes=900 sources=%s\n" % sha)
    got, note = bench.profile_traffic("k_local_d8", 400)
    assert got == 3600 and "scaled" in note
    (csrc / "fr_d8.cu").write_text("// changed\n")
    got, note = bench.profile_traffic("k_local_d8", 400)
    assert got is None and "changed" in note


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                         timeout=600, cwd=str(ROOT))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "cells/s"
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    assert "32768x32768" in d["config"]["workload"]
