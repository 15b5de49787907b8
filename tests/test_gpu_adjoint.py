"""Adjoint solve and gradients (workload c5: L = sum (u - u_t)^2).

lambda = A^-T dL/du by AIRG on A^T (built from the GPU transpose), checked
against the oracle's dense adjoint (LU of A^T) on 64x64; the autograd
gradients dL/dg = B^T lambda and dL/ds = h lambda checked against central
finite differences on seeded directions.  u is affine in (g, s), so L is
quadratic and central differences carry no truncation error: only rounding
and solver tolerance.
"""
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


def _solver(w):
    vx, vy = velocity(w["theta"])
    return G.AdvectionSolver(w["nx"], w["ny"], vx, vy,
                             opts=G.airg_options_default(**w["opts"])), vx, vy


def test_adjoint_matches_dense_adjoint_64():
    w = workload("c5", 64)
    sv, vx, vy = _solver(w)
    g = torch.tensor(w["g"][0], device="cuda")
    s = torch.tensor(w["s"][0], device="cuda", dtype=torch.float32)
    u = sv.solve_plain(g, s, rtol=1e-12)
    rhs = 2.0 * (u - torch.tensor(w["ut"], device="cuda"))
    lam, info = G.airg_solve_adjoint(sv.handle, rhs, rtol=1e-12)
    assert info.converged
    po = O.advection_2d(64, 64, vx, vy)
    lam_d = O.dense_adjoint(po.A, rhs.cpu().numpy())
    lg = lam.cpu().numpy()
    assert np.linalg.norm(lg - lam_d) / np.linalg.norm(lam_d) <= 1e-9
    # the adjoint hierarchy is AIRG on A^T: its residual is small in the
    # transposed operator
    assert np.linalg.norm(po.A.to_dense().T @ lg - rhs.cpu().numpy()) <= 1e-11 * np.linalg.norm(rhs.cpu().numpy())
    # gradient mapping = transpose of the right-hand-side assembly
    gg, gs = G.airg_rhs_adjoint_advection2d(sv.prob, lam)
    d = abs(vx) + abs(vy)
    assert np.allclose(gg.cpu().numpy(), d * lg[po.inflow], rtol=1e-15, atol=0)
    exp_s = po.h * lg
    exp_s[po.inflow] = 0.0
    assert np.allclose(gs.cpu().numpy(), exp_s, rtol=1e-15, atol=0)


def _exact(po, g, s, order):
    """Exact discrete solution (substitution in upwind order, Sec. 1.1)."""
    return O.sweep_solve(po.A, O.assemble_rhs(po, g, s), order)


def _central(po, order, g, s, ut, dg, ds, step):
    """Central difference of L = sum (u - u_t)^2 at exact solutions along
    (dg, ds): (L(+) - L(-)) / (2 step), with L(+) - L(-) evaluated as
    sum (u+ - u-)(u+ + u- - 2 u_t); also w = (u+ - u-) / (2 step)."""
    up = _exact(po, g + step * dg, s + step * ds, order)
    um = _exact(po, g - step * dg, s - step * ds, order)
    w = (up - um) / (2 * step)
    return float(np.sum(w * (up + um - 2 * ut))), w


@pytest.mark.parametrize("size", [256, 1024])
def test_gradients_match_central_differences_of_the_exact_loss(size):
    """dL/dg and dL/ds from the adjoint AIRG solve against central
    differences of L at exact solutions.  u is affine in (g, s), so L is
    quadratic and the central difference equals the directional derivative
    for every step: the step of 1 leaves only the rounding of the exact
    solutions (~1e-15 relative), while the configured step of 1e-6 divides
    that rounding by 1e-6 (the substitution's accumulated rounding, ~1e-14
    relative per node, becomes ~1e-8 per term), so along dg it must agree
    with the step-1 value to 1e-8 of the sum of the terms' magnitudes.
    The analytic side carries the errors of both solves.  With w_d =
    A^-1 B d = (u+ - u-) / (2 step), the forward solution's error e_u
    enters <dL/dg, d> as 2 <e_u, w_d>, and the adjoint's, lambda + delta
    with A^T delta = -rho (rho its true residual), as -<rho, w_d>, at most
    ||rho|| ||w_d||.  dL/dg (FP64) must stay within 2 |<e_u, w_d>| +
    ||rho|| ||w_d|| + 1e-11 |fd| on every direction, and within 1e-8
    relative.  dL/ds is returned in the FP32 of s,
    so its bound adds the FP32 rounding of each entry, 2^-24 sum
    |gs_i ds_i|."""
    w = workload("c5", size)
    sv, vx, vy = _solver(w)
    g = torch.tensor(w["g"][0], device="cuda", requires_grad=True)
    s32 = torch.tensor(w["s"][0], device="cuda", dtype=torch.float32, requires_grad=True)
    ut = w["ut"]
    rtol = 1e-13
    u = sv.solve(g, s32, rtol)
    L = ((u - torch.tensor(ut, device="cuda")) ** 2).sum()
    L.backward()
    gg = g.grad.cpu().numpy()
    gs = s32.grad.double().cpu().numpy()
    assert s32.grad.dtype == torch.float32
    # the same adjoint solve as the backward pass, for its true residual
    rhs = 2.0 * (u.detach() - torch.tensor(ut, device="cuda"))
    lam, info = G.airg_solve_adjoint(sv.handle, rhs, rtol=rtol)
    assert info.converged
    gg2, _ = G.airg_rhs_adjoint_advection2d(sv.prob, lam)
    assert np.array_equal(gg2.cpu().numpy(), gg)
    rho = info.rel_residual * float(torch.linalg.vector_norm(rhs))
    po = O.advection_2d(size, size, vx, vy)
    order = O.sweep_order(po)
    g0 = w["g"][0]
    s0 = s32.detach().double().cpu().numpy()
    u0 = _exact(po, g0, s0, order)
    e_u = u.detach().cpu().numpy() - u0
    zg, zs = np.zeros_like(g0), np.zeros_like(s0)
    ndir = 32 if size == 1024 else 8
    rel = []
    for k in range(ndir):
        dg, ds = w["dirs_g"][k], w["dirs_s"][k]
        fd, wd = _central(po, order, g0, s0, ut, dg, zs, 1.0)
        fd6, _ = _central(po, order, g0, s0, ut, dg, zs, 1e-6)
        scale = float(np.sum(np.abs(wd * 2 * (u0 - ut))))   # size of the terms of the sum
        assert abs(fd6 - fd) <= 1e-8 * scale, ("step 1e-6", k, fd6, fd, scale)
        an = float(gg @ dg)
        bound = 2 * abs(float(e_u @ wd)) + rho * float(np.linalg.norm(wd)) + 1e-11 * abs(fd)
        assert abs(fd - an) <= bound, ("g direction", k, fd, an, bound)
        rel.append(abs(fd - an) / abs(fd))
        fd, wd = _central(po, order, g0, s0, ut, zg, ds, 1.0)
        an = float(gs @ ds)
        bound = (2 * abs(float(e_u @ wd)) + rho * float(np.linalg.norm(wd))
                 + 2.0 ** -24 * float(np.sum(np.abs(gs * ds))) + 1e-11 * abs(fd))
        assert abs(fd - an) <= bound, ("s direction", k, fd, an, bound)
    assert max(rel) <= 1e-8, rel


@pytest.mark.parametrize("size", [256, 1024])
def test_autograd_gradients_match_differences_of_gpu_solves(size):
    """End to end: central differences of L through the GPU's own forward
    solves (rtol 1e-13).  Their solution error divided by the step 1e-6
    limits the agreement to ~1e-6 relative."""
    w = workload("c5", size)
    sv, vx, vy = _solver(w)
    g = torch.tensor(w["g"][0], device="cuda", requires_grad=True)
    s32 = torch.tensor(w["s"][0], device="cuda", dtype=torch.float32, requires_grad=True)
    ut = torch.tensor(w["ut"], device="cuda")
    rtol = 1e-13
    u = sv.solve(g, s32, rtol)
    L = ((u - ut) ** 2).sum()
    L.backward()
    gg = g.grad.double()
    gs = s32.grad.double()
    assert s32.grad.dtype == torch.float32
    s64 = s32.detach().double()
    eps = 1e-6
    ndir = 32 if size == 1024 else 8
    errs = []
    with torch.no_grad():
        for k in range(ndir):
            dg = torch.tensor(w["dirs_g"][k], device="cuda")
            ds = torch.tensor(w["dirs_s"][k], device="cuda")
            lp = ((sv.solve_plain(g.detach() + eps * dg, s64 + eps * ds, rtol) - ut) ** 2).sum()
            lm = ((sv.solve_plain(g.detach() - eps * dg, s64 - eps * ds, rtol) - ut) ** 2).sum()
            fd = float((lp - lm) / (2 * eps))
            an = float((gg * dg).sum() + (gs * ds).sum())
            errs.append(abs(fd - an) / abs(an))
    # FP32 storage of dL/ds limits the analytic side to ~1e-7 relative
    assert max(errs) <= 2e-5, errs
    assert np.median(errs) <= 2e-6, errs
