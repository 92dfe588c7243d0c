"""The bench's roofline bookkeeping on the CPU: the ALU peaks from unit counts, the roofline
fraction (F32/P32 + F64/P64) / time of the algorithmic per-update counts, and the DRAM traffic
record, which holds only while the step kernel's sources are the ones it was captured from."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_alu_peaks_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x FMA (2 flop) x 2.07 GHz; 2 FP64 FMA per SM per clock
    assert abs(bench.FP32_PEAK_TFLOPS - 80.54784) < 1e-9
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-9


def test_roofline_fraction_of_the_algorithmic_counts():
    nodes, K = 262144, 2.0
    f32_node = 800.0 * 16 * K + 1000.0           # per update: 16 populations x K iterations
    f64_node = 150.0 * K + 50.0
    t_roof = nodes * (f32_node / 80.54784e12 + f64_node / 1.25856e12)
    f32, f64, frac = bench.roofline_terms(nodes, K, 2.0 * t_roof)
    assert abs(f32 - nodes * f32_node) < 1e-3 and abs(f64 - nodes * f64_node) < 1e-3
    assert abs(frac - 0.5) < 1e-12
    # at the headline's measured 260 us per launch the fraction is about 0.61
    assert 0.60 < bench.roofline_terms(nodes, K, 260e-6)[2] < 0.62


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    key = "step_kernel_fp32_batched_4x256x256"
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[key]
    assert bench.profiled_traffic(key) == rec["bytes_per_launch"]
    assert rec["bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    # the same record over a copy of the sources with one byte changed is not used
    fake = tmp_path / "root"
    for f in rec["sources"]:
        dst = fake / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, f), "rb").read())
    (fake / "profiles").mkdir()
    (fake / "profiles" / "traffic.json").write_text(json.dumps({key: rec}))
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.profiled_traffic(key) == rec["bytes_per_launch"]
    src = fake / rec["sources"][0]
    src.write_bytes(src.read_bytes() + b" ")
    assert bench.profiled_traffic(key) is None
    assert bench.profiled_traffic("no_such_kernel") is None
