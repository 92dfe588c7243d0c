"""The bench's roofline bookkeeping on the CPU: the ALU peaks from unit counts, the SM count
and a clock, the algorithmic per-update counts, the roofline fraction (F32 + F64) / P / time
with all the work charged to the pipe that executes it, and the DRAM traffic record, which
holds only while the step kernel's sources are the ones it was captured from."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_alu_peaks_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x FMA (2 flop) x 2.07 GHz; 2 FP64 FMA per SM per clock
    p32, p64 = bench.pipe_peaks(152, 2070.0)
    assert abs(p32 - 80.54784) < 1e-9
    assert abs(p64 - 1.25856) < 1e-9
    # the peaks follow the SM count and the clock they are given
    q32, q64 = bench.pipe_peaks(76, 1035.0)
    assert abs(q32 - p32 / 4) < 1e-9 and abs(q64 - p64 / 4) < 1e-9


def test_algorithmic_counts():
    K = 2.0
    f32, f64 = bench.algorithmic_flops(1, K)                    # cubic 2-D D2Q16
    assert f32 == 800.0 * 16 * K + 1000.0 and f64 == 150.0 * K + 50.0
    f32, _ = bench.algorithmic_flops(1, K, taps=3)              # 3-point 2-D: 9 taps
    assert f32 == (2 * 20 * 9 + 160.0) * 16 * K + 1000.0
    f32, _ = bench.algorithmic_flops(1, K, taps=3, one_d=True)  # quasi-1-D: x taps only
    assert f32 == (2 * 20 * 3 + 160.0) * 16 * K + 1000.0
    assert bench.algorithmic_flops(10, K)[0] == 10 * bench.algorithmic_flops(1, K)[0]


def test_roofline_fraction_charges_every_flop_to_one_pipe():
    nodes, K = 262144, 2.0
    f32, f64 = bench.algorithmic_flops(nodes, K)
    p32, _ = bench.pipe_peaks(152, 2070.0)
    t_roof = (f32 + f64) / (p32 * 1e12)
    assert abs(bench.roofline_fraction(f32, f64, 2.0 * t_roof, p32) - 0.5) < 1e-12
    # at 258.7 us per launch (the last measured headline launch) the FP32-pipe fraction is
    # about 0.34; the old two-pipe sum F32/P32 + F64/P64 gave 0.62 for the same launch
    assert 0.33 < bench.roofline_fraction(f32, f64, 258.7e-6, p32) < 0.35


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    """A record is used only while the sources it names hash to its sources_sha256: on a copy
    of the sources with the record's hash recomputed it is used, after a one-byte change it
    is not.  (The committed record itself may be stale: then the bench reports null.)"""
    import hashlib
    key = "step_kernel_fp32_batched_4x256x256"
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[key]
    assert rec["bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    live = bench.profiled_traffic(key)
    assert live is None or live == rec["bytes_per_launch"]
    fake = tmp_path / "root"
    h = hashlib.sha256()
    for f in rec["sources"]:
        dst = fake / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        data = open(os.path.join(ROOT, f), "rb").read()
        dst.write_bytes(data)
        h.update(data)
    rec = dict(rec, sources_sha256=h.hexdigest())
    (fake / "profiles").mkdir()
    (fake / "profiles" / "traffic.json").write_text(json.dumps({key: rec}))
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.profiled_traffic(key) == rec["bytes_per_launch"]
    src = fake / rec["sources"][0]
    src.write_bytes(src.read_bytes() + b" ")
    assert bench.profiled_traffic(key) is None
    assert bench.profiled_traffic("no_such_kernel") is None


def test_clock_summary_keeps_the_timed_region():
    """Samples before the region (warm-up, autotuning) are dropped; the region's own samples
    and the first one after its end are kept, and throttle reasons among them are reported."""
    clk = bench.ClockSampler(0)

    def line(mhz, thermal="Not Active", power="Not Active"):
        return "0, %d, 2070, 900.0, 0x0, Not Active, Not Active, %s, %s" % (mhz, thermal, power)

    clk.stamped = [(0.00, line(1200, thermal="Active")),   # before the region
                   (0.10, line(2070)), (0.15, line(2060, power="Active")),
                   (0.30, line(2050)),                        # first after the end
                   (0.40, line(900))]                         # later: ignored
    clk.t0, clk.t1 = 0.05, 0.20
    c = clk.summary()
    assert c["samples"] == 3 and c["sm_mhz"] == 2060.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    # a region shorter than the sampling interval keeps the sample that closes it
    clk.t0, clk.t1 = 0.16, 0.18
    c = clk.summary()
    assert c["samples"] == 1 and c["sm_mhz"] == 2050.0
    # nothing sampled at all
    clk.stamped = []
    assert bench.ClockSampler.summary(clk)["reasons"] == ["unsampled"]
