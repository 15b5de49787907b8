"""Invalid inputs are rejected with a status, not a fault: every case below is
caught either on the host or by the validation kernel before any entry
outside [0, nnz) is read, and a valid setup and solve work right after."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2508_17517_gb300 as G  # noqa: E402
from synthetic import velocity, workload  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()


def _good(nx=24, ny=20):
    w = workload("grid", (nx, ny))
    vx, vy = velocity(w["theta"])
    pg = G.airg_problem_advection2d(nx, ny, vx, vy)
    return pg["rowptr"].clone(), pg["col"].clone(), pg["val"].clone()


def _status(rowptr, col, val, opts=None):
    with pytest.raises(G.AirgError) as e:
        G.airg_setup(rowptr, col, val, opts)
    return e.value.status


@pytest.mark.parametrize("device", [True, False])
def test_bad_row_pointers(device):
    rp, c, v = _good()
    rp[-1] += 5                                  # rowptr[n] beyond nnz
    if not device:
        rp, c, v = rp.cpu(), c.cpu(), v.cpu()
    assert _status(rp, c, v) == 1
    rp, c, v = _good()
    rp[7] = rp[8] + 1                            # decreasing
    if not device:
        rp, c, v = rp.cpu(), c.cpu(), v.cpu()
    assert _status(rp, c, v) == 1
    rp, c, v = _good()
    rp[3] = -4                                   # negative
    if not device:
        rp, c, v = rp.cpu(), c.cpu(), v.cpu()
    assert _status(rp, c, v) == 1


def test_bad_columns_diagonal_and_values():
    rp, c, v = _good()
    a = int(rp[40])
    c2 = c.clone()
    c2[a] = 10**6                                # column out of range
    assert _status(rp, c2, v) == 1
    assert "columns" in G.airg_last_error()
    c2 = c.clone()
    lo, hi = int(rp[41]), int(rp[42])
    assert hi - lo >= 2
    c2[lo], c2[lo + 1] = c[lo + 1], c[lo]        # not ascending
    assert _status(rp, c2, v) == 1
    # drop the diagonal of row 50 by making it point at a neighbour column
    lo, hi = int(rp[50]), int(rp[51])
    cols = c[lo:hi].cpu().numpy()
    assert 50 in cols and hi - lo >= 2
    v2 = v.clone()
    v2[lo + int(np.nonzero(cols == 50)[0][0])] = float("nan")
    assert _status(rp, c, v2) == 1               # non-finite value
    assert "finite" in G.airg_last_error()
    c_host = c.cpu().numpy()
    keep = [k for k in range(int(rp[-1])) if not (lo <= k < hi and c_host[k] == 50)]
    rp3 = rp.clone()
    rp3[51:] -= 1
    assert _status(rp3, c[keep].contiguous(), v[keep].contiguous()) == 1
    assert "diagonal" in G.airg_last_error()


def test_bad_shapes_and_options():
    rp, c, v = _good()
    n = rp.numel() - 1
    A = G.airg_csr(n, n + 1, c.numel(), rp.data_ptr(), c.data_ptr(), v.data_ptr(), 1)
    out = ctypes.c_void_p()
    o = G.airg_options_default()
    assert G.lib().airg_setup(ctypes.byref(A), ctypes.byref(o), None, ctypes.byref(out)) == 1
    for field, bad in [("gmres_restart", 0), ("gmres_restart", 31), ("precision", 7), ("outer", 3)]:
        assert _status(rp, c, v, G.airg_options_default(**{field: bad})) == 1
    info = G.airg_solve_info()
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st = G.lib().airg_solve(None, 1, b.data_ptr(), x.data_ptr(), 1, 1e-10, 1e-50, 100,
                            ctypes.byref(info), None)
    assert st != 0


def test_valid_solve_after_errors():
    rp, c, v = _good(40, 33)
    rp_bad = rp.clone()
    rp_bad[-1] += 1
    assert _status(rp_bad, c, v) == 1
    h = G.airg_setup(rp, c, v)
    b = torch.ones(rp.numel() - 1, dtype=torch.float64, device="cuda")
    x, info = G.airg_solve(h, b, rtol=1e-10)
    assert info.converged and info.rel_residual <= 1e-10


def test_degenerate_inputs():
    """Edge cases of the problem itself: an empty operator is rejected; the
    single-node system (one inflow node, Eq. 2) solves to u = g; a zero
    right-hand side returns x = 0 at once, for one and for several
    right-hand sides; maxit = 0 returns x0 as not converged."""
    e_rp = torch.zeros(1, dtype=torch.int64, device="cuda")
    e_c = torch.zeros(0, dtype=torch.int32, device="cuda")
    e_v = torch.zeros(0, dtype=torch.float64, device="cuda")
    assert _status(e_rp, e_c, e_v) == 1
    # the grid builder needs two nodes per side; a single inflow node is the
    # 1 x 1 system d u = d g, passed as a CSR matrix
    with pytest.raises(G.AirgError):
        G.airg_problem_advection2d(1, 1, 0.6, 0.8)
    d = 1.4
    h = G.airg_setup(torch.tensor([0, 1], dtype=torch.int64, device="cuda"),
                     torch.tensor([0], dtype=torch.int32, device="cuda"),
                     torch.tensor([d], dtype=torch.float64, device="cuda"))
    x, info = G.airg_solve(h, torch.tensor([d * 0.75], dtype=torch.float64, device="cuda"), rtol=1e-12)
    assert info.converged and abs(float(x[0]) - 0.75) <= 1e-15
    rp, c, v = _good(33, 29)
    h = G.airg_setup(rp, c, v)
    n = rp.numel() - 1
    x, info = G.airg_solve(h, torch.zeros(n, dtype=torch.float64, device="cuda"), rtol=1e-10)
    assert info.converged and info.iterations == 0 and not bool(x.any())
    X, info = G.airg_solve(h, torch.zeros(3, n, dtype=torch.float64, device="cuda"), rtol=1e-10)
    assert info.converged and not bool(X.any())
    # maxit = 0 with a nonzero right-hand side: nothing to do, reported as not converged
    x, info = G.airg_solve(h, torch.ones(n, dtype=torch.float64, device="cuda"), rtol=1e-10, maxit=0,
                           allow_nc=True)
    assert not info.converged and not bool(x.any())
