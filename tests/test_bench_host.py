"""Host-side measurement arithmetic of bench.py (CPU): the dominant kernel's
roofline, the step-level HBM fraction, the committed-traffic lookup keyed by the
kernel's source hash, and the nvidia-smi clock summary.  No GPU, no library."""
import json
import os

import pytest

import bench


def stat(name, launches, total_ms, flops, nbytes, tensor):
    return {"name": name, "launches": launches, "total_ms": total_ms, "flops": flops,
            "bytes": nbytes, "tensor": tensor}


@pytest.fixture
def root(tmp_path, monkeypatch):
    """bench.ROOT pointed at an empty tree (no peaks file, no traffic records)."""
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def write_peaks(root, **peaks):
    with open(root / "MEASURED_PEAKS.json", "w") as f:
        json.dump(peaks, f)


def test_alu_peak_is_sms_lanes_fma_clock():
    assert bench.alu_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert bench.alu_peak_tflops(1000.0) == pytest.approx(38.912)


def test_roofline_takes_the_kernel_with_the_largest_time_against_the_measured_peaks(root):
    write_peaks(root, hbm_gbs=6000.0, bf16_tflops_sustained=1500.0, sm_max_mhz=2000.0)
    stats = [stat("fwd axis0+1 tc32 mid", 4, 8.0, 4e12, 8e9, True),
             stat("fwd axis2 lagsum-tcgen05-1024 last", 4, 12.0, 24e12, 16e9, True),
             stat("inv axis0 reg16 last", 1, 0.1, 1e9, 1e8, False)]
    r = bench.roofline(stats, "nowhere", "mixed", profiled_units=4 * 2048)
    assert r["kernel"] == "fwd axis2 lagsum-tcgen05-1024 last"
    assert r["bound"] == "tensor" and r["peak"] == 1500.0
    # 6e12 flops per launch in 3 ms = 2000 TFLOP/s; 4e9 bytes in 3 ms = 1333.3 GB/s
    assert r["avg_launch_ms"] == pytest.approx(3.0)
    assert r["achieved"] == pytest.approx(2000.0)
    assert r["frac"] == pytest.approx(2000.0 / 1500.0, abs=1e-4)
    assert r["hbm"]["achieved"] == pytest.approx(1333.3, abs=0.1)
    assert r["hbm"]["frac"] == pytest.approx(1333.33 / 6000.0, abs=1e-4)
    assert r["share_of_kernel_time"] == pytest.approx(12.0 / 20.1, abs=1e-4)
    assert "of measured" in r["peak_note"]
    assert r["traffic"] is None  # no record for this workload


def test_roofline_alu_bound_kernel_and_the_serial_figures(root):
    write_peaks(root, hbm_gbs=6780.4, sm_max_mhz=2070.0)
    stats = [stat("fwd axis1 smem3x2048 last", 2, 2.0, 30e9, 2e9, False)]
    serial = [stat("fwd axis1 smem3x2048 last", 2, 1.0, 30e9, 2e9, False)]
    r = bench.roofline(stats, "nowhere", "fp32", serial_stats=serial, serial_shares={"fwd axis1 smem3x2048 last": 0.6})
    alu = bench.alu_peak_tflops(2070.0)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(round(alu, 1))
    assert r["achieved"] == pytest.approx(15.0)  # 15e9 flops in 1 ms
    assert r["serial"]["avg_launch_ms"] == pytest.approx(0.5)
    assert r["serial"]["achieved"] == pytest.approx(30.0)
    assert r["serial"]["hbm_achieved"] == pytest.approx(2000.0)
    assert r["share_serial"] == 0.6


def test_roofline_falls_back_without_the_peaks_file(root):
    r = bench.roofline([stat("fwd axis2 lagsum-tcgen05-1024 last", 1, 1.0, 1.7e12, 1e9, True)], "nowhere", "mixed")
    assert r["peak"] == 1700.0 and "of fallback" in r["peak_note"]
    assert r["hbm"]["peak"] == 6800.0
    assert bench.roofline([stat("x", 0, 0.0, 0, 0, False)], "nowhere", "fp32") is None


def test_step_hbm_divides_a_steps_algorithmic_bytes_by_its_time(root):
    write_peaks(root, hbm_gbs=5000.0)
    stats = [stat("a", 2, 1.0, 0, 6e9, False), stat("b", 2, 1.0, 0, 4e9, False)]
    s = bench.step_hbm(stats, 2.0)  # bytes over bench.PROFILED_STEPS steps
    per_step = 10e9 / bench.PROFILED_STEPS
    assert s["bytes_per_step"] == pytest.approx(per_step)
    assert s["achieved"] == pytest.approx(per_step / 2e-3 / 1e9, abs=0.1)
    assert s["frac"] == pytest.approx(per_step / 2e-3 / 1e9 / 5000.0, abs=1e-4)
    assert bench.step_hbm(stats, 0) is None


def test_traffic_record_is_used_only_while_the_kernel_sources_match(root):
    name = "fwd axis1 smem3x2048 last"
    h = bench.kernel_source_hash(name)
    assert len(h) == 16 and h != bench.kernel_source_hash("fwd axis2 lagsum-tcgen05-1024 last")
    with open(root / "profiles" / "traffic.txt", "w") as f:
        f.write("# comment | not | a | record | 1 | 1\n")
        f.write(f"grid1024 | fp32 | {name} | {h} | 1000000 | 64\n")
        f.write(f"grid1024 | fp32 | fwd axis0 smem3x2048 mid | 0000000000000000 | 5 | 64\n")
    assert bench.recorded_traffic(name, "grid1024", "fp32", 64) == (1000000.0, "ncu, same launch size")
    b, note = bench.recorded_traffic(name, "grid1024", "fp32", 128)
    assert b == pytest.approx(2000000.0) and "scaled" in note
    # another workload or precision, or a stale hash: no figure
    assert bench.recorded_traffic(name, "hier2", "fp32", 64) == (None, None)
    assert bench.recorded_traffic(name, "grid1024", "mixed", 64) == (None, None)
    assert bench.recorded_traffic("fwd axis0 smem3x2048 mid", "grid1024", "fp32", 64) == (None, None)


def test_source_hash_covers_the_pass_kinds_own_files():
    # kinds sharing one source file share a hash; the generic prefixes do not
    # swallow the more specific ones listed before them
    assert bench.kernel_source_hash("fwd axis2 lagsum-tcgen05-1024 last") == \
        bench.kernel_source_hash("fwd axis2 xspec-tcgen05-64 last")
    assert bench.kernel_source_hash("fwd axis2 lagsum-tcgen05-bf16-1024 last") == \
        bench.kernel_source_hash("fwd axis2 lagsum-tcgen05-1024 last")
    assert bench.kernel_source_hash("fwd axis2 xspec64 last") != \
        bench.kernel_source_hash("fwd axis2 xspec-tcgen05-64 last")
    assert bench.kernel_source_hash("fwd axis1 smem3x2048 last") != \
        bench.kernel_source_hash("fwd axis1 smem2048 last")
    assert bench.kernel_source_hash("fwd axis0+1 tc32 mid") != \
        bench.kernel_source_hash("fwd axis2+3 tcgen05-16 last")


def test_committed_traffic_records_are_well_formed():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.txt")) as f:
        rows = [l for l in f if l.strip() and not l.startswith("#")]
    assert rows
    for l in rows:
        p = [v.strip() for v in l.split("|")]
        assert len(p) == 6, l
        assert p[1] in ("fp32", "mixed", "mixed_bf16"), l
        int(p[3], 16)
        assert len(p[3]) == 16 and float(p[4]) > 0 and float(p[5]) > 0, l


def test_clock_summary_median_max_and_active_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1900, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "0, 2060, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "garbage line\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path = object(), str(path)
    s = cs.summary()
    assert s == {"sm_mhz": 2060.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not path.exists()
    assert bench.ClockSampler(0).summary() is None
