"""Host-side pieces of bench.py that need no GPU: the DRAM-traffic lookup, the roofline
denominators and the algorithmic byte / flop tables."""
import json
import os

import bench


def test_traffic_entries_are_well_formed():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    csrc = os.listdir(os.path.join(bench.ROOT, "paper_1407_6486_gb300", "csrc"))
    for key, e in d.items():
        if key.startswith("_"):
            continue
        kernel, n = key.split("@")
        assert int(n) > 0 and e["bytes_per_point"] > 0
        assert all(f in csrc for f in e["src_files"]), key
        # the lookup returns the stored value exactly when the kernel's sources are unchanged
        current = bench.kernel_src_hash(e["src_files"]) == e["src_hash"]
        got = bench.traffic_for(kernel, int(n))
        assert (got == e["bytes_per_point"]) if current else got is None


def test_traffic_lookup_ignores_unknown_kernels():
    assert bench.traffic_for("no_such_kernel", 255) is None


def test_fp64_peak_is_the_unit_count_times_the_clock():
    assert abs(bench.FP64_NOMINAL_GFLOPS - 152 * 2.07 * 4) < 1e-9


def test_algorithmic_bytes_of_the_fine_kernels():
    # FP32 multigrid data (t = 4): sweep reads e and f and writes e; the update sweep adds
    # the FP64 read-modify-write of u; the pointwise residual reads two FP64 values
    assert bench.algo_bytes_per_point("rbgs_sweep3d", 4) == 12
    assert bench.algo_bytes_per_point("rbgs_sweep3d_upd", 4) == 24
    assert bench.algo_bytes_per_point("resid_pt", 4) == 20
    assert bench.algo_fp64_flops_per_point("fine_rhs_residual", 5, 3) == 84
