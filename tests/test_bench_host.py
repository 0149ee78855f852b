"""Host-side logic of bench.py that needs no GPU: the staleness rule of the committed
traffic figures, the peak denominators, the launch count of a graph-driven form and
the clock summary."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_tree(tmp_path, src=b"__global__ void k() {}\n"):
    csrc = tmp_path / "paper_2203_13675_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_bytes(src)
    (tmp_path / "profiles").mkdir()
    return csrc


def test_traffic_is_used_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    csrc = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    assert len(h) == 16
    prof = tmp_path / "profiles" / "fcg_mixed_mg_U_c2_2048.txt"
    prof.write_text(f"header\nsource_hash: {h}\ndram_bytes_per_px_iter: 25.31\n")
    assert bench.profile_traffic("fcg_mixed_mg_U_c2_2048") == 25.31
    # any change to a CUDA source makes the summary stale: no traffic is reported
    (csrc / "k.cu").write_bytes(b"__global__ void k() { }\n")
    assert bench.kernel_source_hash() != h
    assert bench.profile_traffic("fcg_mixed_mg_U_c2_2048") is None
    assert bench.profile_traffic("missing_profile") is None


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == (6800.0, "fallback")
    allp = bench.load_peaks_all()
    assert allp["hbm"] == (6800.0, "fallback") and allp["bf16"][0] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps(
        {"hbm_gbs": 6682.8, "bf16_tflops": 1886.9, "bf16_tflops_sustained": 1732.9}))
    assert bench.load_peaks() == (6682.8, "measured")
    allp = bench.load_peaks_all()
    assert allp["hbm"][0] == 6682.8 and allp["bf16"][0] == 1886.9 and allp["bf16_sust"][0] == 1732.9


def test_graph_form_launch_count():
    # host launches, plus per timed step and outer pass: the start kernels and one loop
    # body per inner iteration
    cnt = {"kernel_launches": 10, "graph_start_kernels": 7, "graph_body_kernels": 16}
    st = {"inner": [37, 7, 4, 3, 3]}
    assert bench.gpu_launches(cnt, st, ("mixed", "mg"), 3) == 10 + 3 * (5 * 7 + 54 * 16)
    # a persistent form counts its host launches only
    assert bench.gpu_launches(cnt, st, ("f64", "jacobi"), 3) == 10


def test_clock_summary_flags_throttle_reasons():
    c = bench.ClockSampler(None)
    c.lines = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]
