"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Setup products must match bit for bit: CF splitting, every sparsity pattern
and, by construction (fixed operation order, correctly rounded dots), every
value.  The coarse-grid roots come from two different eigenvalue solvers and
are compared with a tolerance.  Solutions must agree with the oracle to
1e-9 relative L2 at rtol 1e-10, with the true residual at or below rtol.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2508_17517_gb300 as G  # noqa: E402
from oracle import airg as O  # noqa: E402
from synthetic import velocity, workload  # noqa: E402

pytestmark = pytest.mark.gpu
T_ROOT = __import__("os").path.dirname(__import__("os").path.dirname(__import__("os").path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()


def _oopts(d):
    o = {k: v for k, v in d.items() if k not in ("precision", "outer", "smoother", "smooth_type", "inverse_type")}
    if d.get("smoother", 0) == 1:
        o["smoother"] = "assembled"
    o["smooth_type"] = ("f", "fc", "fcf")[d.get("smooth_type", 0)]
    o["inverse_type"] = ("gmres", "neumann")[d.get("inverse_type", 0)]
    return O.Options(**o)


def _csr_equal(M, exp, what, exact_values=True):
    nr, nc, rp, ci, v = exp
    assert (nr, nc) == (M.n_rows, M.n_cols), what
    assert np.array_equal(rp, M.rowptr), what + " rowptr"
    assert np.array_equal(ci.astype(np.int64), M.col), what + " pattern"
    if exact_values:
        bad = np.nonzero(v != M.val)[0]
        assert bad.size == 0, "%s values differ at %d entries, max rel %.3e" % (
            what, bad.size, np.max(np.abs(v[bad] - M.val[bad]) / np.maximum(np.abs(M.val[bad]), 1e-300)))


class Case:
    def __init__(self, w, opts_over=None):
        self.w = w
        o = dict(w["opts"])
        o.update(opts_over or {})
        self.o = o
        vx, vy = velocity(w["theta"])
        self.po = O.advection_2d(w["nx"], w["ny"], vx, vy)
        self.pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
        self.Ho = O.setup(self.po.A, _oopts(o))
        self.h = G.airg_setup(self.pg["rowptr"], self.pg["col"], self.pg["val"],
                              G.airg_options_default(**o))


def _check_setup(c):
    Ho, h = c.Ho, c.h
    info = G.airg_setup_info(h)
    assert info["levels"] == len(Ho.levels) + 1
    assert info["truncated"] == Ho.truncated
    for l, L in enumerate(Ho.levels):
        cf = G.airg_export_vector(h, l, 0).astype(bool)
        assert np.array_equal(cf, L.is_f), "CF split level %d" % l
        _csr_equal(L.A, G.airg_export_matrix(h, l, 0), "A_%d" % l)
        _csr_equal(L.A_ff, G.airg_export_matrix(h, l, 1), "A_ff level %d" % l)
        _csr_equal(L.A_fc, G.airg_export_matrix(h, l, 2), "A_fc level %d" % l)
        _csr_equal(L.Z, G.airg_export_matrix(h, l, 3), "Z level %d" % l)
        assert np.array_equal(G.airg_export_vector(h, l, 1), L.W), "W level %d" % l
        assert np.array_equal(G.airg_export_vector(h, l, 2), L.alpha), "alpha level %d" % l
        if L.A_cc is not None:
            _csr_equal(L.A_cc, G.airg_export_matrix(h, l, 5), "A_cc level %d" % l)
        if L.Ainv_cc is not None:
            _csr_equal(L.Ainv_cc, G.airg_export_matrix(h, l, 6), "Ahat_cc^-1 level %d" % l)
            assert np.array_equal(G.airg_export_vector(h, l, 5), L.alpha_c), "alpha_c level %d" % l
        sc = G.airg_export_vector(h, l, 4)
        assert int(sc[0]) == L.pmisr_rounds
        assert [int(x) for x in sc[1:-2]] == list(L.ddc_converted)
    _csr_equal(Ho.A_coarse, G.airg_export_matrix(h, len(Ho.levels), 0), "A_coarse")
    # Roots come from two eigen-solvers; eigenvalues of a non-normal
    # Hessenberg are ill-conditioned, so compare what matters: the number of
    # roots (same Krylov dimension) and the polynomial they define, applied
    # by the oracle to a random vector.
    r = G.airg_export_vector(h, len(Ho.levels), 3).reshape(-1, 2)
    ro = np.array(Ho.roots)
    assert r.shape[0] >= 1 and abs(r.shape[0] - ro.shape[0]) <= 2
    assert info["coarse_krylov"] == Ho.coarse_k
    v = np.random.default_rng(7).standard_normal(Ho.A_coarse.n_rows)
    qg = O.newton_apply(Ho.A_coarse, [tuple(x) for x in r], v)
    qo = O.newton_apply(Ho.A_coarse, Ho.roots, v)
    assert np.linalg.norm(qg - qo) <= 1e-6 * np.linalg.norm(qo)


def _check_solve(c, rtol=None, host=False):
    w = c.w
    rtol = rtol or w["rtol"]
    s = w["s"][0] if w["s"] is not None else np.zeros(c.po.A.n_rows)
    bo = O.assemble_rhs(c.po, w["g"][0], s)
    gt = torch.tensor(w["g"][0], device="cuda")
    st = torch.tensor(s, device="cuda")
    bg = G.airg_assemble_rhs_advection2d(c.pg, gt, st)
    assert np.array_equal(bg.cpu().numpy(), bo)
    xo, io = O.solve(c.Ho, c.po.A, bo, rtol=rtol)
    if host:
        bh = torch.tensor(bo)
        xg, ig = G.airg_solve(c.h, bh, rtol=rtol)
        xg = xg.numpy()
    else:
        xg, ig = G.airg_solve(c.h, bg, rtol=rtol)
        xg = xg.cpu().numpy()
    res = np.linalg.norm(bo - O.spmv(c.po.A, xg)) / np.linalg.norm(bo)
    assert ig.converged and res <= rtol * (1 + 1e-6)
    rel = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert rel <= 1e-9, "GPU vs oracle rel L2 %.3e" % rel
    u = O.sweep_solve(c.po.A, bo, O.sweep_order(c.po))
    assert np.linalg.norm(xg - u) / np.linalg.norm(u) <= 1e-9
    return xg, ig, io


def _check_one_cycle(c, tol):
    """One FGMRES step from x0 = 0 returns x_1 = c M^-1 b with the scalar c
    fixed by the least-squares problem, so comparing x_1 with the oracle's
    compares one V-cycle application itself (a converged solution would hide
    a weaker preconditioner)."""
    s = c.w["s"][0] if c.w["s"] is not None else np.zeros(c.po.A.n_rows)
    bo = O.assemble_rhs(c.po, c.w["g"][0], s)
    xo, _ = O.solve(c.Ho, c.po.A, bo, rtol=1e-300, maxit=1)
    xg, _ = G.airg_solve(c.h, torch.tensor(bo, device="cuda"), rtol=1e-300, maxit=1, allow_nc=True)
    rel = np.linalg.norm(xg.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert rel <= tol, "one V-cycle: GPU vs oracle rel L2 %.3e" % rel


# ------------------------------------------------------------ primitives --
def test_exact_dot_bitwise():
    rng = np.random.default_rng(0)
    for n in [1, 7, 1000, 100003, 3_000_001]:
        x = rng.standard_normal(n) * np.exp2(rng.integers(-40, 40, n))
        y = rng.standard_normal(n)
        got = G.airg_dot_exact(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"))
        assert got == O.xdot(x, y)
    assert G.airg_dot_exact(torch.zeros(5, device="cuda", dtype=torch.float64),
                            torch.ones(5, device="cuda", dtype=torch.float64)) == 0.0
    # magnitudes that keep a thread's products in one digit window, that
    # walk the window up and down, extreme and subnormal exponents, and
    # exact cancellation
    n = 1 << 21
    cases = [(rng.uniform(0.5, 1.0, n), rng.uniform(-1.0, 1.0, n)),
             (np.exp2(np.linspace(-60, 60, n)), rng.standard_normal(n)),
             (np.exp2(np.linspace(60, -60, n)), rng.standard_normal(n)),
             (rng.standard_normal(n) * np.exp2(rng.integers(-1000, 1000, n)), rng.standard_normal(n)),
             (rng.standard_normal(4099) * 1e-310, rng.standard_normal(4099))]
    z = rng.standard_normal(n // 2)
    cases.append((np.concatenate([z, z]), np.concatenate([z, -z])))
    for x, y in cases:
        got = G.airg_dot_exact(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"))
        assert got == O.xdot(x, y)


def test_rng_bitwise():
    for lev, pur, n in [(0, 1, 10), (3, 2, 100001), (7, 4, 1)]:
        g = G.airg_rng_uniform(2508175, lev, pur, n).cpu().numpy()
        assert np.array_equal(g, O.rng_uniform(2508175, lev, pur, n))


@pytest.mark.parametrize("theta", [3 * math.pi / 8, 0.0, math.pi / 2 + 0.3, 3.7, 5.5])
def test_builder_bitwise(theta):
    vx, vy = velocity(theta)
    po = O.advection_2d(37, 23, vx, vy)
    pg = G.airg_problem_advection2d(37, 23, vx, vy)
    assert np.array_equal(pg["rowptr"].cpu().numpy(), po.A.rowptr)
    assert np.array_equal(pg["col"].cpu().numpy().astype(np.int64), po.A.col)
    assert np.array_equal(pg["val"].cpu().numpy(), po.A.val)
    assert np.array_equal(pg["inflow"].cpu().numpy(), po.inflow)


# ----------------------------------------------------------- full paths --
def test_c1_setup_and_solve():
    c = Case(workload("c1"))
    _check_setup(c)
    _check_one_cycle(c, 1e-12)
    xg, ig, io = _check_solve(c)
    assert np.max(np.abs(xg - 1.0)) < 1e-8          # Eq. 1-2: u = g = 1
    assert abs(ig.iterations - io.iterations) <= 1


@pytest.mark.parametrize("shape", [(203, 157), (96, 331)])
def test_ragged_grids(shape):
    c = Case(workload("grid", shape))
    _check_setup(c)
    _check_one_cycle(c, 1e-12)
    _check_solve(c)


@pytest.mark.parametrize("name,shape", [("hard", (150, 150)), ("rect", (30, 1200))])
def test_hard_direction_and_rectangle(name, shape):
    """The paper's other studies at oracle size: v = (sqrt(2/3), sqrt(1/3))
    with strong threshold 0.4 (Sec. 3.3.2), and a long thin rectangle at
    pi/4 with coarse order 10 (Sec. 3.4)."""
    c = Case(workload(name, shape))
    _check_setup(c)
    _check_solve(c)
    _check_one_cycle(c, 1e-12)


def test_host_buffer_path():
    c = Case(workload("grid", (120, 90)))
    _check_solve(c, host=True)


def test_grid_aligned_exact():
    w = workload("grid", (48, 40))
    w["theta"] = 0.0
    w["g"] = np.random.default_rng(1).random((1, 40))
    c = Case(w, dict(trunc_rtol=0.0, coarse_min_rows=40))
    _check_setup(c)
    xg, ig, io = _check_solve(c)
    assert ig.iterations <= 2


def test_pure_polynomial_and_level0_truncation():
    w = workload("grid", (40, 40))
    c = Case(w, dict(max_levels=1, coarse_poly_order=100))
    _check_setup(c)
    _check_solve(c)
    c2 = Case(w, dict(trunc_rtol=0.5, coarse_poly_order=100))
    _check_setup(c2)
    assert c2.Ho.truncated


def test_tiny_grid():
    c = Case(workload("grid", (2, 3)))
    _check_setup(c)
    _check_solve(c)


def test_mixed_precision_fp32_vcycle():
    w = workload("grid", (256, 200))
    c = Case(w, dict(precision=1))
    _check_setup(c)
    _check_solve(c)


def test_c2_full_size():
    """The 1024x1024 workload of the benchmark, complete comparison."""
    c = Case(workload("c2"))
    _check_setup(c)
    _check_solve(c)


@pytest.mark.parametrize("env", [("AIRG_NO_GRAPHS", "1"), ("AIRG_PERSISTENT", "1"),
                                 ("AIRG_PERSISTENT", "coarse"), ("AIRG_PERSISTENT", "smoother")])
def test_alternative_launch_paths(env, monkeypatch):
    """Direct kernel launches (no CUDA graph) and the persistent cooperative
    polynomial kernels (coarse Newton and/or F smoother, one launch each with
    a bounded grid barrier) give the same parity as the default path."""
    monkeypatch.setenv(*env)
    c = Case(workload("grid", (160, 120)))
    _check_solve(c)


@pytest.mark.parametrize("n,prec", [(1024, 0), (2048, 1)])
def test_coarse_steps_with_x_in_shared_memory(n, prec, monkeypatch):
    """The coarse Newton steps with x staged in shared memory
    (AIRG_COARSE_XS=1) give the same bits as the unstaged steps
    (AIRG_COARSE_XS=0): they compute every row with the same summation
    order.  1024^2 in FP64 (17k coarse rows of ~170 entries, 8 warps per
    slice, the last slice ragged) and 2048^2 with the FP32 V-cycle."""
    w = workload("c2", n)
    vx, vy = velocity(w["theta"])
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    opts = G.airg_options_default(**dict(w["opts"], precision=prec))
    b = G.airg_assemble_rhs_advection2d(pg, torch.tensor(w["g"][0], device="cuda"))
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("AIRG_COARSE_XS", mode)
        h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"], opts)
        info = G.airg_setup_info(h)
        nco, nnz = info["n"][info["levels"] - 1], info["nnz_a"][info["levels"] - 1]
        x, si = G.airg_solve(h, b, rtol=w["rtol"])
        out[mode] = (x, si.iterations, si.rel_residual)
    # the staged form applies: long rows (several warps per slice) and x fits
    # in shared memory beside the 32 x 32 reduction tile
    vb = 8 if prec == 0 else 4
    assert nnz / nco > 24 and nco * vb + 32 * 32 * vb <= 227 * 1024, (nco, nnz)
    (x0, it0, rr0), (x1, it1, rr1) = out["0"], out["1"]
    assert it0 == it1 and rr0 == rr1
    assert torch.equal(x0, x1)
    assert rr1 <= w["rtol"]


def test_chunked_sparse_products(monkeypatch):
    """Sparse products split into many row chunks (tiny hash-table budget)
    give the same bits as in one chunk."""
    monkeypatch.setenv("AIRG_SPGEMM_SLOTS", "4096")
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r); import tests.test_gpu_parity as T; "
            "from synthetic import workload; c = T.Case(workload('grid', (150, 130))); "
            "T._check_setup(c); T._check_solve(c)" % T_ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]


def test_bounded_device_wait_reports_timeout():
    """A device-side wait that nothing satisfies gives up after its poll
    limit and reports AIRG_ERR_TIMEOUT; the context stays usable."""
    assert G.airg_check_wait_timeout(20000) == 6
    assert "gave up" in G.airg_last_error()
    c = Case(workload("grid", (40, 30)))
    _check_solve(c)


@pytest.mark.parametrize("prec", [0, 1])
def test_richardson_outer_matches_oracle(prec):
    """Outer Richardson (Sec. 3): same iteration count as the oracle's
    Richardson on the same hierarchy, solution within 1e-9 of both the
    oracle and the sweep."""
    w = workload("grid", (150, 131))
    c = Case(w, {"outer": G.AIRG_OUTER_RICHARDSON, "precision": prec})
    s = w["s"][0]
    bo = O.assemble_rhs(c.po, w["g"][0], s)
    bg = G.airg_assemble_rhs_advection2d(c.pg, torch.tensor(w["g"][0], device="cuda"),
                                         torch.tensor(s, device="cuda"))
    xo, io = O.solve(c.Ho, c.po.A, bo, rtol=1e-10, outer="richardson")
    xg, ig = G.airg_solve(c.h, bg, rtol=1e-10)
    xg = xg.cpu().numpy()
    assert ig.converged and io.converged
    assert abs(ig.iterations - io.iterations) <= (0 if prec == 0 else 1)
    assert np.linalg.norm(bo - O.spmv(c.po.A, xg)) <= 1e-10 * np.linalg.norm(bo) * (1 + 1e-6)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-9
    u = O.sweep_solve(c.po.A, bo, O.sweep_order(c.po))
    assert np.linalg.norm(xg - u) / np.linalg.norm(u) <= 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_slices_per_warp_never_changes_a_bit(prec, monkeypatch):
    """The setup's timing-based choices -- slices per warp (1, 2 or 4) for
    short rows, loads in flight per lane (4, 8 or 16) for long rows, the
    operator's own grid or a resident grid striding over the slices -- only
    change how rows are mapped to threads: forcing each choice gives the
    same solution bit for bit."""
    w = workload("grid", (300, 257))
    vx, vy = velocity(w["theta"])
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    b = G.airg_assemble_rhs_advection2d(pg, torch.tensor(w["g"][0], device="cuda"),
                                        torch.tensor(w["s"][0], device="cuda"))
    xs = []
    for r, u, pg_ in [("1", "4", "0"), ("2", "8", "0"), ("4", "16", "0"), ("1", "4", "1"), ("4", "16", "1")]:
        monkeypatch.setenv("AIRG_ROWS_PER_WARP", r)
        monkeypatch.setenv("AIRG_LOADS_PER_LANE", u)
        monkeypatch.setenv("AIRG_PERSIST_GRID", pg_)
        h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"],
                         G.airg_options_default(precision=prec, **w["opts"]))
        x, info = G.airg_solve(h, b, rtol=1e-10)
        assert info.converged
        xs.append(x.cpu().numpy())
    for x in xs[1:]:
        assert np.array_equal(xs[0], x)


@pytest.mark.parametrize("prec", [0, 1])
def test_16bit_columns_never_change_a_bit(prec, monkeypatch):
    """16-bit column indices (the index itself for the coarsest operator,
    with at most 65536 columns; the offset from each slice's smallest column
    for the level and top-level operators, whose 409,600 columns need the
    slice bases) hold the same values as the 32-bit ones: solutions are
    equal bit for bit with and without them, at every slices-per-warp and
    loads-per-lane setting of the row kernels, and with the coarse steps
    streaming the operator through shared memory by bulk copies."""
    w = workload("c2", n=640)
    vx, vy = velocity(w["theta"])
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    b = G.airg_assemble_rhs_advection2d(pg, torch.tensor(w["g"][0], device="cuda"))
    xs, vbytes = [], []
    for col16, r, u, stream in [("0", "1", "4", "0"), ("1", "1", "4", "0"), ("1", "2", "8", "0"),
                                ("1", "4", "16", "0"), ("1", "1", "4", "1")]:
        monkeypatch.setenv("AIRG_COL16", col16)
        monkeypatch.setenv("AIRG_ROWS_PER_WARP", r)
        monkeypatch.setenv("AIRG_LOADS_PER_LANE", u)
        monkeypatch.setenv("AIRG_COARSE_STREAM", stream)
        h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"],
                         G.airg_options_default(precision=prec, **w["opts"]))
        info = G.airg_setup_info(h)
        assert info["n"][-1] <= 65536
        vbytes.append(info["bytes_per_vcycle"])
        x, si = G.airg_solve(h, b, rtol=1e-10)
        assert si.converged
        xs.append(x.cpu().numpy())
    # the 16-bit paths were taken: fewer index bytes per V-cycle
    assert vbytes[1] < vbytes[0] and vbytes[1] == vbytes[2] == vbytes[3] == vbytes[4]
    for x in xs[1:]:
        assert np.array_equal(xs[0], x)


@pytest.mark.parametrize("prec", [0, 1])
def test_serpentine_order_never_changes_a_bit(prec, monkeypatch):
    """The chains of SpMVs with one operator (the Horner terms of a level,
    the coarse Newton steps) alternate their traversal direction; with
    AIRG_SERPENTINE=0 every step runs forward.  Each row is computed the
    same way either way, so the solutions are equal bit for bit, for the
    F-point and the FC smoother (whose C-point Horner chain alternates
    too)."""
    w = workload("c2", n=384)
    vx, vy = velocity(w["theta"])
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    b = G.airg_assemble_rhs_advection2d(pg, torch.tensor(w["g"][0], device="cuda"))
    for smoother in (0, 1):
        xs = []
        for serp in ("0", "1"):
            monkeypatch.setenv("AIRG_SERPENTINE", serp)
            h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"],
                             G.airg_options_default(precision=prec, smooth_type=smoother, **w["opts"]))
            x, si = G.airg_solve(h, b, rtol=1e-10)
            assert si.converged
            xs.append(x.cpu().numpy())
        assert np.array_equal(xs[0], xs[1])


def test_bf16_restrictor_storage_error():
    """Restrictor values in bfloat16 (FP32 V-cycle): the outer FP64 iteration
    still meets rtol and the solution matches the oracle and the sweep to
    1e-9; the cost of the narrower R is reported as extra iterations, at
    most two over the FP32 V-cycle."""
    w = workload("grid", (257, 300))
    vx, vy = velocity(w["theta"])
    po = O.advection_2d(w["nx"], w["ny"], vx, vy)
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    bo = O.assemble_rhs(po, w["g"][0], w["s"][0])
    b = torch.tensor(bo, device="cuda")
    u = O.sweep_solve(po.A, bo, O.sweep_order(po))
    Ho = O.setup(po.A, _oopts(w["opts"]))
    xo, io = O.solve(Ho, po.A, bo, rtol=1e-10)
    its = {}
    for prec in [G.AIRG_FP64, G.AIRG_MIXED_FP32, G.AIRG_MIXED_FP32_BF16R]:
        h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"], G.airg_options_default(precision=prec, **w["opts"]))
        x, info = G.airg_solve(h, b, rtol=1e-10)
        xg = x.cpu().numpy()
        assert info.converged
        assert np.linalg.norm(bo - O.spmv(po.A, xg)) <= 1e-10 * np.linalg.norm(bo) * (1 + 1e-6)
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-9
        assert np.linalg.norm(xg - u) / np.linalg.norm(u) <= 1e-9
        its[prec] = info.iterations
    assert its[G.AIRG_MIXED_FP32_BF16R] <= its[G.AIRG_MIXED_FP32] + 2, its



@pytest.mark.parametrize("prec", [0, 1])
def test_assembled_smoother_matches_oracle(prec):
    """Smoother = the assembled fixed-sparsity matrix of Eq. 8 (Sec. 2.2):
    the stored matrices equal the oracle's bit for bit, and the solve matches
    the oracle's solve with the same smoother and the sweep to 1e-9."""
    w = workload("grid", (170, 143))
    c = Case(w, {"smoother": G.AIRG_SMOOTH_ASSEMBLED, "precision": prec})
    _check_setup(c)
    for l, L in enumerate(c.Ho.levels):
        _csr_equal(L.Ainv, G.airg_export_matrix(c.h, l, 4), "Ahat^-1 level %d" % l)
    _check_one_cycle(c, 1e-12 if prec == 0 else 1e-4)
    _check_solve(c)


@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("smooth_type", [1, 2])
def test_c_point_smoothing_matches_oracle(smooth_type, prec, smoother):
    """FC and FCF smoothing (Sec. 2, the options of Sec. 3.3.2): A_cc and the
    C-point polynomial bit for bit, the solution within 1e-9 of the oracle
    (FP64 and FP32 V-cycles), and the complexities of the extra blocks."""
    w = workload("grid", (203, 157))
    c = Case(w, dict(smooth_type=smooth_type, precision=prec, smoother=smoother))
    _check_setup(c)
    xg, ig, io = _check_solve(c)
    # the preconditioner itself must match, not only the converged solution
    _check_one_cycle(c, 1e-12 if prec == 0 else 1e-4)
    assert abs(ig.iterations - io.iterations) <= (1 if prec == 0 else 2), (ig.iterations, io.iterations)
    cf = G.airg_setup_info(G.airg_setup(c.pg["rowptr"], c.pg["col"], c.pg["val"],
                                        G.airg_options_default(smoother=smoother, **w["opts"])))
    cs = G.airg_setup_info(c.h)
    extra = sum(L.A.nnz - L.A_ff.nnz - L.A_fc.nnz + (L.Ainv_cc.nnz if L.Ainv_cc is not None else 0)
                for L in c.Ho.levels)
    assert abs((cs["storage_complexity"] - cf["storage_complexity"]) * c.po.A.nnz - extra) < 1e-6 * c.po.A.nnz
    assert cs["cycle_complexity"] > cf["cycle_complexity"]


@pytest.mark.parametrize("smoother", [0, 1])
def test_c_point_smoothing_many_rhs_and_grids(smoother):
    """FCF smoothing in the batched many-RHS V-cycle and in a batch of grids:
    one V-cycle (a single outer step from zero) and the converged solutions
    match the oracle for every right-hand side."""
    w = workload("grid", (90, 70))
    opts = dict(w["opts"], smooth_type=2, smoother=smoother)
    vx, vy = velocity(w["theta"])
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    po = O.advection_2d(w["nx"], w["ny"], vx, vy)
    Ho = O.setup(po.A, _oopts(opts))
    h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"], G.airg_options_default(**opts))
    B = torch.rand(3, w["nx"] * w["ny"], dtype=torch.float64, device="cuda",
                   generator=torch.Generator("cuda").manual_seed(5))
    X1, _ = G.airg_solve(h, B, rtol=1e-300, maxit=1, allow_nc=True)
    X, _ = G.airg_solve(h, B, rtol=1e-10)
    for q in range(3):
        bo = B[q].cpu().numpy()
        x1, _ = O.solve(Ho, po.A, bo, rtol=1e-300, maxit=1)
        assert np.linalg.norm(X1[q].cpu().numpy() - x1) <= 1e-12 * np.linalg.norm(x1)
        xo, _ = O.solve(Ho, po.A, bo, rtol=1e-10)
        xg = X[q].cpu().numpy()
        assert np.linalg.norm(bo - O.spmv(po.A, xg)) <= 1e-10 * np.linalg.norm(bo) * (1 + 1e-6)
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-9
    w2 = workload("grid", (61, 77))
    vx2, vy2 = velocity(w2["theta"])
    pg2 = G.airg_problem_advection2d(w2["nx"], w2["ny"], vx2, vy2)
    po2 = O.advection_2d(w2["nx"], w2["ny"], vx2, vy2)
    Bt = G.airg_setup_batch([(pg["rowptr"], pg["col"], pg["val"]), (pg2["rowptr"], pg2["col"], pg2["val"])],
                            G.airg_options_default(**opts))
    bs = [B[0].contiguous(), torch.ones(w2["nx"] * w2["ny"], dtype=torch.float64, device="cuda")]
    xs, infos = G.airg_solve_batch(Bt, bs, rtol=1e-10)
    for x, b, P in zip(xs, bs, (po, po2)):
        Hp = O.setup(P.A, _oopts(opts))
        xo, _ = O.solve(Hp, P.A, b.cpu().numpy(), rtol=1e-10)
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-9

@pytest.mark.parametrize("prec", [0, 1])
def test_nair_matches_oracle(prec):
    """nAIR (Sec. 3.3.1): the Neumann coefficients bit for bit (they decide
    Z and every coarse operator), the hierarchy bit for bit, and the solution
    within 1e-9 of the oracle; the batched many-RHS form agrees too."""
    w = workload("grid", (203, 157))
    c = Case(w, dict(inverse_type=1, precision=prec))
    _check_setup(c)
    xg, ig, io = _check_solve(c)
    _check_one_cycle(c, 1e-12 if prec == 0 else 1e-4)
    assert abs(ig.iterations - io.iterations) <= (1 if prec == 0 else 2), (ig.iterations, io.iterations)
    B = torch.rand(4, w["nx"] * w["ny"], dtype=torch.float64, device="cuda",
                   generator=torch.Generator("cuda").manual_seed(9))
    X, _ = G.airg_solve(c.h, B, rtol=1e-10)
    for q in range(4):
        bo = B[q].cpu().numpy()
        xo, _ = O.solve(c.Ho, c.po.A, bo, rtol=1e-10)
        xg = X[q].cpu().numpy()
        assert np.linalg.norm(bo - O.spmv(c.po.A, xg)) <= 1e-10 * np.linalg.norm(bo) * (1 + 1e-6)
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-9
