"""The committed ncu records the benchmark reports beside its roofline cover
the current sources of the headline workload's frame kernels, in either form
the autotuner may pick (one launch, or pass 1 + pass 2); they turn stale, and
this fails, when those sources change without a new capture.  A record
applies only to its own kernel and workload."""
import pytest

import bench


KERNEL = "k_frame_unit"   # the octree frame's kernel in one launch


@pytest.mark.parametrize("kernel", ["k_frame_unit", "k_pass1_unit_frame", "k_pass2_unit_frame"])
def test_ncu_record_matches_current_kernel_sources(kernel):
    rec = bench.measured_ncu(kernel, "amr")
    assert rec is not None, f"profiles/ record of {kernel} is stale: re-capture it"
    assert rec["dram_bytes_per_launch"] > 1e8 and rec["samples_per_launch"] > 1e8
    assert 0 < rec["issue_active_pct"] <= 100 and 0 < rec["l1_data_pipe_pct"] <= 100
    assert bench.measured_traffic(kernel, "amr") == int(rec["dram_bytes_per_launch"])


def test_ncu_record_is_not_reused_for_other_kernels_or_workloads():
    assert bench.measured_ncu("k_pass2_unit", "amr") is None          # the split form has no record
    assert bench.measured_ncu(KERNEL, "tets") is None
    assert bench.measured_traffic(KERNEL, "tets") is None
    one = bench.measured_ncu(KERNEL, "amr")
    two = bench.measured_ncu("k_pass1_unit_frame", "amr")
    assert one["launch_ms"] != two["launch_ms"]


def test_ncu_record_round_trip(tmp_path):
    """The record writer reads an ncu raw CSV dump and the reader takes it
    back only for the same kernel, workload and sources."""
    csv = tmp_path / "raw.csv"
    names = ["dram__bytes_read.sum", "dram__bytes_write.sum", "smsp__inst_executed.sum", "gpu__time_duration.sum",
             "smsp__issue_active.avg.pct_of_peak_sustained_active", "sm__throughput.avg.pct_of_peak_sustained_elapsed",
             "l1tex__throughput.avg.pct_of_peak_sustained_active", "lts__throughput.avg.pct_of_peak_sustained_elapsed",
             "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed",
             "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active",
             "sm__inst_executed_pipe_fma.avg.pct_of_peak_sustained_active",
             "sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active",
             "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active"]
    units = ["Gbyte", "Mbyte", "inst", "msecond"] + ["%"] * 9
    vals = ["1.5", "500", "3200000", "2.0"] + ["50"] * 9
    csv.write_text("\n".join(",".join(f'"{x}"' for x in row) for row in (names, units, vals)) + "\n")
    old = bench.NCU_DIR
    try:
        bench.NCU_DIR = str(tmp_path)
        out = tmp_path / "ncu_k_test_blobs64.txt"
        rec = bench.write_ncu_record(str(csv), "k_test", "blobs64", 400000, str(out))
        assert rec["dram_bytes_per_launch"] == 2_000_000_000 and rec["inst_per_sample"] == 256.0
        back = bench.measured_ncu("k_test", "blobs64")
        assert back["dram_bytes_per_launch"] == 2e9 and back["samples_per_launch"] == 400000
        assert bench.measured_ncu("k_other", "blobs64") is None
    finally:
        bench.NCU_DIR = old


def test_roofs_pick_the_largest_fraction():
    """The four roofs of a launch: ALU and MUFU from the algorithmic counts
    and the launch time (here chosen so that ALU is at 25 % and MUFU at 50 %
    of their peaks), HBM from the DRAM bytes at 10 % of the copy rate, L2 from
    the record's percentage; the binding roof is the largest of them, and a
    roof without data is left out of the choice."""
    samples, ms = 1.0e9, 10.0
    flop = 0.25 * bench.FP32_PEAK_TFLOPS * 1e12 * ms * 1e-3 / samples
    mufu = 0.5 * bench.MUFU_PEAK_TOPS * 1e12 * ms * 1e-3 / samples
    hbm_gbs = 6000.0
    traffic = 0.1 * hbm_gbs * 1e9 * ms * 1e-3
    rec = {"l2_throughput_pct": 30.0, "issue_active_pct": 71.0}
    r = bench.roofs_of(samples, ms, flop, mufu, traffic, hbm_gbs, rec)
    assert r["alu_frac"] == pytest.approx(0.25) and r["mufu_frac"] == pytest.approx(0.5)
    assert r["hbm_frac"] == pytest.approx(0.1) and r["l2_frac"] == pytest.approx(0.3)
    assert r["binding"] == "mufu" and r["binding_frac"] == pytest.approx(0.5)
    assert r["issue_active_frac_ncu"] == pytest.approx(0.71)
    bare = bench.roofs_of(samples, ms, 4 * flop, mufu, None, hbm_gbs, None)
    assert bare["hbm_frac"] is None and bare["l2_frac"] is None
    assert bare["binding"] == "alu" and bare["binding_frac"] == pytest.approx(1.0)
