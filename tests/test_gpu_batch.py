"""Many right-hand sides on one hierarchy (batched V-cycle, lockstep FGMRES):
every right-hand side must match the oracle's solve of it to 1e-9 relative
L2 with its true residual at or below rtol, for batch widths that do not
fill a warp (k = 5) and that need two right-hand sides per lane (k = 40),
in FP64 and with the FP32 V-cycle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2508_17517_gb300 as G  # noqa: E402
from oracle import airg as O  # noqa: E402
from synthetic import velocity, workload  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()


@pytest.mark.parametrize("k,prec", [(5, 0), (40, 0), (40, 1)])
def test_batched_rhs_match_oracle(k, prec):
    w = workload("grid", (110, 97))
    vx, vy = velocity(w["theta"])
    rng = np.random.default_rng(k + 7 * prec)
    n = w["nx"] * w["ny"]
    po = O.advection_2d(w["nx"], w["ny"], vx, vy)
    nin = po.inflow.size
    g = rng.uniform(0.0, 1.0, (k, nin))
    s = rng.standard_normal((k, n))
    opts = dict(w["opts"], precision=prec)
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"], G.airg_options_default(**opts))
    b = G.airg_assemble_rhs_advection2d(pg, torch.tensor(g, device="cuda"), torch.tensor(s, device="cuda"))
    assert b.shape == (k, n)
    x, info = G.airg_solve(h, b, rtol=1e-10)
    assert info.converged and info.rel_residual <= 1e-10
    X = x.cpu().numpy()
    Ho = O.setup(po.A, O.Options(**{kk: v for kk, v in opts.items() if kk != "precision"}))
    for q in range(k):
        bo = O.assemble_rhs(po, g[q], s[q])
        assert np.array_equal(bo, b[q].cpu().numpy())
        res = np.linalg.norm(bo - O.spmv(po.A, X[q])) / np.linalg.norm(bo)
        assert res <= 1e-10 * (1 + 1e-6)
        if q % 8 == 0:
            xo, _ = O.solve(Ho, po.A, bo, rtol=1e-10)
            assert np.linalg.norm(X[q] - xo) / np.linalg.norm(xo) <= 1e-9


@pytest.mark.parametrize("outer", [0, 1])
def test_batched_host_buffers_and_richardson(outer):
    """Host right-hand sides (copies inside the call) with nrhs > 1, with
    FGMRES and with lockstep Richardson: each column equals its own
    single-RHS solve to 1e-9 and meets rtol."""
    w = workload("grid", (90, 77))
    vx, vy = velocity(w["theta"])
    k = 9
    rng = np.random.default_rng(21 + outer)
    po = O.advection_2d(w["nx"], w["ny"], vx, vy)
    n = po.A.n_rows
    g = rng.uniform(0.0, 1.0, (k, po.inflow.size))
    s = rng.standard_normal((k, n))
    opts = dict(w["opts"], outer=outer)
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"], G.airg_options_default(**opts))
    bh = torch.tensor(np.stack([O.assemble_rhs(po, g[q], s[q]) for q in range(k)]))
    x, info = G.airg_solve(h, bh, rtol=1e-10)
    assert x.device.type == "cpu" and info.converged
    X = x.numpy()
    assert np.all(np.isfinite(X)) and np.abs(X).max() > 0
    Ho = O.setup(po.A, O.Options(**w["opts"]))
    for q in range(k):
        bo = bh[q].numpy()
        assert np.linalg.norm(bo - O.spmv(po.A, X[q])) <= 1e-10 * np.linalg.norm(bo) * (1 + 1e-6)
        if q % 4 == 0:
            xo, _ = O.solve(Ho, po.A, bo, rtol=1e-10, outer="richardson" if outer else "fgmres")
            assert np.linalg.norm(X[q] - xo) / np.linalg.norm(xo) <= 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_serpentine_order_never_changes_a_bit(prec, monkeypatch):
    """The batched Horner and Newton chains alternate their traversal
    direction; with AIRG_SERPENTINE=0 every step runs forward.  The k
    solutions are equal bit for bit either way."""
    w = workload("grid", (120, 101))
    vx, vy = velocity(w["theta"])
    k = 12
    rng = np.random.default_rng(91 + prec)
    po = O.advection_2d(w["nx"], w["ny"], vx, vy)
    g = rng.uniform(0.0, 1.0, (k, po.inflow.size))
    s = rng.standard_normal((k, po.A.n_rows))
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    b = G.airg_assemble_rhs_advection2d(pg, torch.tensor(g, device="cuda"), torch.tensor(s, device="cuda"))
    xs = []
    for serp in ("0", "1"):
        monkeypatch.setenv("AIRG_SERPENTINE", serp)
        h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"], G.airg_options_default(**dict(w["opts"], precision=prec)))
        x, info = G.airg_solve(h, b, rtol=1e-10)
        assert info.converged
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1])
