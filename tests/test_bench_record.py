"""The committed ncu record the benchmark reports beside its roofline covers
the current sources of the frame kernels (it turns stale, and this fails,
when those sources change without a new capture), and applies only to its
own kernel and workload."""
import bench


KERNEL = "k_frame_fused"   # the frame's kernel: one launch per frame


def test_ncu_record_matches_current_kernel_sources():
    rec = bench.measured_ncu(KERNEL, "blobs512")
    assert rec is not None, "profiles/ record is stale: re-capture the frame kernel"
    assert rec["dram_bytes_per_launch"] > 1e9
    assert 0 < rec["issue_active_pct"] <= 100 and 0 < rec["l1_data_pipe_pct"] <= 100
    assert bench.measured_traffic(KERNEL, "blobs512") == int(rec["dram_bytes_per_launch"])


def test_ncu_record_is_not_reused_for_other_kernels_or_workloads():
    assert bench.measured_ncu("k_pass2_fused_frame", "blobs512") is None
    assert bench.measured_ncu("k_pass1_fused_frame", "blobs512") is None
    assert bench.measured_ncu(KERNEL, "amr") is None
    assert bench.measured_traffic(KERNEL, "tets") is None
