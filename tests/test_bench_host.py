"""Host logic of bench.py's roofline entry (no GPU): the bound follows the
roofline model, min(peak_BW * intensity, arithmetic peak)."""
import os

import numpy as np

import bench


def test_fp64_dot_products_are_alu_bound():
    # 8 bytes and one FMA (2 flops) per element: 0.25 flop/B * 6.77 TB/s
    # = 1.69 TFLOP/s > 1.26 TFLOP/s FP64 peak
    prof = {"krylov_vectors": (10.0, 100, 8 * 10**10)}
    per = {("krylov_vectors", 0): (10.0, 100, 8 * 10**10, 2 * 10**10)}
    e = bench.roofline_from(prof, per, per[("krylov_vectors", 0)], 1, 20.0, 21.0, 6769.4, "measured")
    assert e["bound"] == "alu" and e["unit"] == "TFLOP/s"
    assert abs(e["achieved"] - 2.0) < 1e-12
    assert e["kernel"] == "krylov_vectors (level 0)"


def test_spmv_is_hbm_bound_and_dominant_group_wins():
    # FP32 SpMV, 8 bytes per stored entry and one FMA: 0.25 flop/B is far
    # below the FP32 peak; the larger of two groups is reported, with the
    # figures of its own timing pass and its share of the uninstrumented step
    prof = {"f_smoother": (12.0, 60, 6 * 10**10), "restrict": (3.0, 10, 10**10)}
    per = {("f_smoother", 0): (8.0, 30, 4 * 10**10, 10**10),
           ("f_smoother", 3): (4.0, 30, 2 * 10**10, 5 * 10**9),
           ("restrict", 0): (3.0, 10, 10**10, 2 * 10**9)}
    assert bench.dominant_group(per) == ("f_smoother", 0)
    alone = (14.0, 60, 8 * 10**10, 2 * 10**10)      # two solves, group timed alone
    e = bench.roofline_from(prof, per, alone, 2, 20.0, 20.5, 6769.4, "measured", "f32")
    assert e["bound"] == "hbm" and e["unit"] == "GB/s"
    assert e["kernel"] == "f_smoother (level 0)"
    assert abs(e["achieved"] - 8 * 10**10 / 14e-3 / 1e9) < 1e-6
    assert abs(e["share"] - 7.0 / 20.0) < 1e-12          # share x ms_per_step = group ms per solve
    assert abs(e["share"] * 20.0 - e["group_ms_per_step"]) < 1e-12
    assert e["dtype"] == "f32"


def test_traffic_lookup_is_tied_to_the_kernel_source(tmp_path, monkeypatch):
    """The roofline's traffic comes from the committed ncu summary only when
    it was measured on the current kernel source; otherwise it is null with
    the reason."""
    src = bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "coarse_newton_traffic.md").write_text(
        "| workload | kind | level | kernel source | launches | algorithmic B per launch | DRAM B per launch | us |\n"
        "|---|---|---|---|---|---|---|---|\n"
        "| c3_fp64 | coarse_newton | 11 | %s | 3 | 1.0e8 | 1.1e8 | 50 |\n"
        "| c3_fp32 | coarse_newton | 11 | 000000000000 | 3 | 5.0e7 | 5.5e7 | 40 |\n" % src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "paper_2508_17517_gb300").symlink_to(
        os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2508_17517_gb300"))
    t, s = bench.measured_traffic("c3_fp64", "coarse_newton", 11)
    assert t == 1.1e8 and s == src
    t, s = bench.measured_traffic("c3_fp64", "coarse_newton", 11, alg_bytes=1.005e8)
    assert t == 1.1e8
    t, s = bench.measured_traffic("c3_fp64", "coarse_newton", 11, alg_bytes=0.9e8)
    assert t is None and "operator" in s
    t, s = bench.measured_traffic("c3_fp32", "coarse_newton", 11)
    assert t is None and "not the current" in s
    t, s = bench.measured_traffic("c2", "f_smoother", 0)
    assert t is None


def test_cpu_baseline_sample_runs_at_least_min_seconds():
    """The oracle baseline repeats whole solves until the sample reaches its
    minimum duration, and reports DOFs per second over all of them."""
    from synthetic import workload
    w = workload("c1")
    v, ts, its, setup_s = bench.cpu_oracle_solve(w, 1, 0, min_seconds=0.05)
    assert len(ts) >= 1 and sum(ts) >= 0.05 and its > 0 and setup_s > 0
    assert abs(v - w["nx"] * w["ny"] * len(ts) / sum(ts)) <= 1e-9 * v
    v2, ts2, _, _ = bench.cpu_oracle_solve(w, 2, 0)
    assert len(ts2) == 2


def test_exact_substitution_context():
    """The serial substitution timed beside the oracle baseline reports the
    DOFs per second of its best run, and its solution is exact (u = 1 for
    constant inflow 1 and no source)."""
    from synthetic import workload
    w = workload("c1")
    u, v, t = bench.cpu_exact(w, repeats=2)
    assert t > 0 and abs(v - w["nx"] * w["ny"] / t) <= 1e-9 * v
    assert np.max(np.abs(u - 1.0)) < 1e-14


def test_reference_sample_of_the_4096_workload_is_its_corner():
    """The oracle's bounded sample of the 4096^2 workloads is the 1024^2
    lower-left corner with the same direction, options and inflow values."""
    from synthetic import workload
    ws, what = bench.reference_sample(bench.parse([]))
    w = workload("c3_fp64")
    assert "corner" in what and ws["nx"] == ws["ny"] == bench.CORNER
    assert ws["theta"] == w["theta"] and ws["opts"] == w["opts"] and ws["rtol"] == w["rtol"]
    m, nx = bench.CORNER, w["nx"]
    assert np.array_equal(ws["g"][0][:m], w["g"][0][:m])
    assert np.array_equal(ws["g"][0][m:], w["g"][0][nx:nx + m - 1])
    ws2, what2 = bench.reference_sample(bench.parse(["--workload", "c2"]))
    assert what2 == "the workload" and ws2["nx"] == 1024


def test_corner_solution_is_the_restriction_of_the_full_solution():
    """Upwind dependence closes the corner: on a small grid of the same
    kind, the exact solution of the corner problem equals the full
    problem's on the corner."""
    from oracle import airg as O
    from synthetic import corner, velocity, workload
    w = workload("c3_fp64", n=48)
    wc = corner(w, 20)
    vx, vy = velocity(w["theta"])
    pf = O.advection_2d(48, 48, vx, vy)
    pc = O.advection_2d(20, 20, vx, vy)
    uf = O.sweep_solve(pf.A, O.assemble_rhs(pf, w["g"][0], np.zeros(48 * 48)), O.sweep_order(pf))
    uc = O.sweep_solve(pc.A, O.assemble_rhs(pc, wc["g"][0], np.zeros(400)), O.sweep_order(pc))
    assert np.array_equal(uf.reshape(48, 48)[:20, :20].reshape(-1), uc)


def test_row_kernel_choices_are_recorded_per_operator():
    """The line's hierarchy.row_kernels: one entry per operator the solve
    keeps, naming its level, warps per slice, r, grid form, index and value
    bytes (16-bit offsets from slice bases marked '+base')."""
    class FakeG:
        @staticmethod
        def airg_row_kernel_choices(h):
            base = dict(n_cols=10, padded=64, dense_diagonal=1)
            return [(0, "top", dict(base, n_rows=1000, nnz=3000, warps_per_slice=1, r=2, resident_grid=1,
                                    index_bytes=4, slice_bases=0, value_bytes=8)),
                    (0, "A_ff", dict(base, n_rows=400, nnz=560, warps_per_slice=1, r=4, resident_grid=0,
                                     index_bytes=2, slice_bases=1, value_bytes=4)),
                    (1, "coarse", dict(base, n_rows=50, nnz=5000, warps_per_slice=8, r=16, resident_grid=0,
                                       index_bytes=2, slice_bases=0, value_bytes=4))]
    rk = bench.row_kernel_choices(FakeG, None)
    assert list(rk) == ["L0 top", "L0 A_ff", "L1 coarse"]
    assert rk["L0 top"] == "1w r2 resident i4 v8, 1000 rows x 3.0"
    assert rk["L0 A_ff"] == "1w r4 own i2+base v4, 400 rows x 1.4"
    assert rk["L1 coarse"] == "8w r16 own i2 v4, 50 rows x 100.0"
    sinfo = {"levels": 2, "n": [1000, 50], "cycle_complexity": 3.0, "storage_complexity": 2.0,
             "bytes_per_vcycle": 1, "setup_ms": 1.0, "setup_breakdown_ms": {"rap": 0.5}, "exact_dots": 0}
    assert "row_kernels" not in bench.hierarchy_entry(sinfo)
    assert bench.hierarchy_entry(sinfo, FakeG, object())["row_kernels"] == rk
