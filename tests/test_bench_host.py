"""Host logic of bench.py's roofline entry (no GPU): the bound follows the
roofline model, min(peak_BW * intensity, arithmetic peak)."""
import bench


def test_fp64_dot_products_are_alu_bound():
    # 8 bytes and one FMA (2 flops) per element: 0.25 flop/B * 6.77 TB/s
    # = 1.69 TFLOP/s > 1.26 TFLOP/s FP64 peak
    prof = {"krylov_vectors": (10.0, 100, 8 * 10**10)}
    per = {("krylov_vectors", 0): (10.0, 100, 8 * 10**10, 2 * 10**10)}
    e = bench.roofline_entry(prof, per, 6769.4, "measured")
    assert e["bound"] == "alu" and e["unit"] == "TFLOP/s"
    assert abs(e["achieved"] - 2.0) < 1e-12
    assert e["kernel"] == "krylov_vectors (level 0)"


def test_spmv_is_hbm_bound_and_dominant_group_wins():
    # FP32 SpMV, 8 bytes per stored entry and one FMA: 0.25 flop/B is far
    # below the FP32 peak; the larger of two groups is reported
    prof = {"f_smoother": (12.0, 60, 6 * 10**10), "restrict": (3.0, 10, 10**10)}
    per = {("f_smoother", 0): (8.0, 30, 4 * 10**10, 10**10),
           ("f_smoother", 3): (4.0, 30, 2 * 10**10, 5 * 10**9),
           ("restrict", 0): (3.0, 10, 10**10, 2 * 10**9)}
    e = bench.roofline_entry(prof, per, 6769.4, "measured", "f32")
    assert e["bound"] == "hbm" and e["unit"] == "GB/s"
    assert e["kernel"] == "f_smoother (level 0)"
    assert abs(e["achieved"] - 4 * 10**10 / 8e-3 / 1e9) < 1e-6
    assert abs(e["share"] - 8.0 / 15.0) < 1e-12
    assert e["dtype"] == "f32"


def test_traffic_table_lookup():
    """The roofline's traffic comes from the committed ncu summary: found for
    the captured (workload, kind, level) groups, absent otherwise."""
    t2 = bench.measured_traffic("c2", "coarse_newton", 8)
    t3 = bench.measured_traffic("c3", "coarse_newton", 11)
    assert t2 is not None and 3e7 < t2 < 5e7
    assert t3 is not None and 1.5e8 < t3 < 2.5e8
    assert bench.measured_traffic("c2", "f_smoother", 0) is None
    assert bench.measured_traffic("c4a", "coarse_newton", 8) is None


def test_many_grid_aggregate_roofline():
    """The many-grid line reports V-cycle bytes over the whole solve's time."""
    e = bench.multi_roofline(6 * 10**9, 2.0, 6769.4, "measured")
    assert e["bound"] == "hbm" and e["unit"] == "GB/s"
    assert abs(e["achieved"] - 3000.0) < 1e-9
    assert abs(e["frac"] - 3000.0 / 6769.4) < 1e-12


def test_cpu_baseline_sample_runs_at_least_min_seconds():
    """The oracle baseline repeats whole solves until the sample reaches its
    minimum duration, and reports DOFs per second over all of them."""
    from synthetic import workload
    w = workload("c1")
    v, ts = bench.cpu_oracle_solve(w, 1, 0, min_seconds=0.05)
    assert len(ts) >= 1 and sum(ts) >= 0.05
    assert abs(v - w["nx"] * w["ny"] * len(ts) / sum(ts)) <= 1e-9 * v
    v2, ts2 = bench.cpu_oracle_solve(w, 2, 0)
    assert len(ts2) == 2


def test_sequential_sweep_context():
    """The serial substitution timed beside the oracle baseline reports the
    DOFs per second of its best run."""
    from synthetic import workload
    w = workload("c1")
    v, t = bench.cpu_sweep(w, repeats=2)
    assert t > 0 and abs(v - w["nx"] * w["ny"] / t) <= 1e-9 * v
