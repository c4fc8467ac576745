"""Host-side bookkeeping of bench.py (CPU only): the roofline arithmetic of a record and the
rule that a recorded DRAM-traffic figure is reported only for the kernel sources it was
measured on."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_instruction_counts():
    # 22 + 3d with loads and the store; 21 + d arithmetic only (degree 3: 31 / 24, 6: 40 / 27)
    assert [bench.alg_instr_per_attempt(d) for d in (3, 6)] == [31, 40]
    assert [bench.alg_instr_arith_only(d) for d in (3, 6)] == [24, 27]


def test_roofline_record_arithmetic():
    # 1e12 attempts in 2 s at 31 instructions each on 152 SMs at 2070 MHz
    rec = bench.roofline(31.0, 24.0, 1e12, 2.0, 152, 2070.0, "no such kernel", "no such workload")
    peak = 152 * 128 * 2070e6 / 1e12
    assert rec["bound"] == "alu" and rec["unit"] == "Tinstr/s"
    assert rec["peak"] == pytest.approx(peak)
    assert rec["achieved"] == pytest.approx(15.5)
    assert rec["frac"] == pytest.approx(15.5 / peak)
    assert rec["frac_arith_only"] == pytest.approx(12.0 / peak)
    assert rec["traffic"] is None and "no ncu capture" in rec["traffic_note"]


def _copy_sources(dst):
    for sub in ("paper_1004_0023_gb300/csrc", "include"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(dst, sub))


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h_sweep, h_batch = bench.kernel_source_hash("sweep"), bench.kernel_source_hash("batch")
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", {("k", "w"): ("sweep", h_sweep, 1234),
                                                      ("b", "w"): ("batch", h_batch, 99)})
    assert bench.measured_traffic("k", "w")[0] == 1234
    assert bench.measured_traffic("b", "w")[0] == 99
    assert bench.measured_traffic("k", "other")[0] is None
    # a change to the sweep kernel's own file makes its figure stale, not the batched one's
    with open(tmp_path / "paper_1004_0023_gb300/csrc/pt_kernels.cu", "a") as f:
        f.write("\n// changed\n")
    nbytes, note = bench.measured_traffic("k", "w")
    assert nbytes is None and note.startswith("stale")
    assert bench.measured_traffic("b", "w")[0] == 99
    # a change to a header both include, or to the public header, makes both stale
    with open(tmp_path / "include/pt.h", "a") as f:
        f.write("\n/* changed */\n")
    assert bench.measured_traffic("b", "w")[0] is None
