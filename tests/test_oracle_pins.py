"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks one oracle step against a closed form, a brute-force or
library computation, an invariant the paper states, or a published value, so
that a dropped term, a wrong sign or index or a transposed operand fails.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import airg as O
from oracle import lib

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(nx, ny, theta):
    return O.advection_2d(nx, ny, math.cos(theta), math.sin(theta))


# ---------------------------------------------------------------- RNG ----
def test_splitmix64_published_outputs():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_1234567.txt"))
            if l.strip() and not l.startswith("#")]
    out = np.empty(len(vals))
    lib().orc_rng_uniform(1234567, len(vals), O._p(out))
    assert [int(v * 2.0 ** 53) for v in out] == [v >> 11 for v in vals]
    u32 = np.empty(len(vals), dtype=np.uint32)
    lib().orc_rng_u32(1234567, len(vals), O._p(u32))
    assert [int(v) for v in u32] == [v >> 32 for v in vals]


def test_rng_streams_distinct_and_uniform():
    a = O.rng_uniform(7, 0, O.PURPOSE_COEF, 20000)
    b = O.rng_uniform(7, 1, O.PURPOSE_COEF, 20000)
    c = O.rng_uniform(7, 0, O.PURPOSE_TRUNC, 20000)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.01


# ------------------------------------------------------ exact dot product --
def _exact_dot(x, y):
    return float(sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)),
                     Fraction(0)))


@pytest.mark.parametrize("case", range(8))
def test_exact_dot_matches_fractions(case):
    rng = np.random.default_rng(case)
    n = [1, 2, 7, 64, 257, 1000, 33, 500][case]
    x = rng.standard_normal(n) * np.exp2(rng.integers(-60, 60, n))
    y = rng.standard_normal(n) * np.exp2(rng.integers(-60, 60, n))
    if case == 6:  # heavy cancellation: sum of products is tiny
        y = np.concatenate([y[: n // 2], -y[: n // 2] * x[: n // 2] / x[n // 2: 2 * (n // 2)], [1e-30]])
        x = np.concatenate([x[: 2 * (n // 2)], [1e-30]])
    assert O.xdot(x, y) == _exact_dot(x, y)


def test_exact_dot_subnormal_and_ties():
    x = np.array([2.0 ** -1074, 2.0 ** -1000, 1.0, 2.0 ** -53])
    y = np.array([1.0, 2.0 ** -60, 1.0, 1.0])
    assert O.xdot(x, y) == _exact_dot(x, y)
    # 1 + 2^-53 is a tie and rounds to even (1.0); adding 2^-1074 breaks the tie upward
    assert O.xdot(np.array([1.0, 2.0 ** -53]), np.array([1.0, 1.0])) == 1.0
    assert O.xdot(np.array([1.0, 2.0 ** -53, 2.0 ** -1074]), np.ones(3)) == 1.0 + 2.0 ** -52
    assert O.xdot(np.zeros(3), np.ones(3)) == 0.0


# ------------------------------------------------------- SpMV / SpGEMM ----
def test_spmv_and_spgemm_against_dense():
    rng = np.random.default_rng(3)
    D = rng.standard_normal((30, 20)) * (rng.random((30, 20)) < 0.2)
    E = rng.standard_normal((20, 25)) * (rng.random((20, 25)) < 0.3)

    def csr(M):
        r, c = np.nonzero(M)
        return O.csr_from_entries(M.shape[0], M.shape[1], r, c, M[r, c])

    A, B = csr(D), csr(E)
    x = rng.standard_normal(20)
    assert np.allclose(O.spmv(A, x), D @ x, rtol=1e-14, atol=1e-14)
    C = O.spgemm(A, B)
    assert np.allclose(C.to_dense(), D @ E, rtol=1e-13, atol=1e-14)
    # pattern of C is the symbolic product pattern
    assert set(zip(C.row_ids(), C.col)) == set(zip(*np.nonzero((D != 0).astype(int) @ (E != 0).astype(int))))
    # integer-valued operands: products and sums are exact
    Di = np.round(D * 4); Ei = np.round(E * 4)
    assert np.array_equal(O.spgemm(csr(Di), csr(Ei)).to_dense(), Di @ Ei)


# --------------------------------------------- problem builder and sweep ----
@pytest.mark.parametrize("theta", [3 * math.pi / 8, math.pi / 4, 0.3, 2.0, 3.5, 5.0])
def test_builder_exact_for_linear_solution(theta):
    """Upwind differences are exact for u = a x + b y + c: with s = v.grad(u)
    and g = u on the inflow edges, the discrete solution is u at the nodes."""
    nx, ny = 17, 11
    P = _grid(nx, ny, theta)
    a, bb, c = 0.7, -1.3, 0.25
    idx = np.arange(nx * ny)
    X = (idx % nx) * P.h
    Y = (idx // nx) * P.h
    u = a * X + bb * Y + c
    s = np.full(nx * ny, P.vx * a + P.vy * bb)
    rhs = O.assemble_rhs(P, u[P.inflow], s)
    sol = O.sweep_solve(P.A, rhs, O.sweep_order(P))
    assert np.max(np.abs(sol - u)) < 1e-12
    # and the dense solve agrees
    assert np.max(np.abs(np.linalg.solve(P.A.to_dense(), rhs) - u)) < 1e-11


def test_builder_structure_c1():
    P = _grid(64, 64, 3 * math.pi / 8)
    A = P.A
    assert A.n_rows == 4096 and P.inflow.size == 127        # 2N-1 inflow nodes
    D = A.to_dense()
    assert np.allclose(D, np.tril(D))                        # lower triangular (Sec. 1.1)
    assert np.all(np.diag(D) == abs(P.vx) + abs(P.vy))
    interior = np.setdiff1d(np.arange(4096), P.inflow)
    assert np.allclose(D[interior].sum(1), 0.0, atol=1e-15)  # consistent: constants in kernel
    assert A.nnz == 4096 + 2 * interior.size


def test_constant_inflow_gives_constant_solution():
    """Eq. 1-2 with constant g and zero source: u = g everywhere."""
    P = _grid(64, 64, 3 * math.pi / 8)
    b = O.assemble_rhs(P, np.full(P.inflow.size, 1.0), np.zeros(4096))
    u = O.sweep_solve(P.A, b, O.sweep_order(P))
    assert np.array_equal(u, np.ones(4096))


# ---------------------------------------------------------------- CF split --
def test_strength_hand_cases():
    P = _grid(8, 8, 3 * math.pi / 8)     # |vy| = 0.924 > |vx| = 0.383: only y-upwind strong
    s = O.strength(P.A, 0.99)
    rid = P.A.row_ids()
    strong_cols = P.A.col[s] - rid[s]
    assert np.all(strong_cols == -8)
    assert s.sum() == 8 * 8 - 15                                  # one per interior row
    P2 = _grid(8, 8, math.pi / 4)        # equal magnitudes: both neighbours strong
    s2 = O.strength(P2.A, 0.99)
    assert s2.sum() == 2 * (64 - 15)
    assert not np.any(s2[P2.A.col == rid])                       # diagonal never strong


def test_strength_hard_direction_threshold():
    """v = (sqrt(2/3), sqrt(1/3)) (Sec. 3.3.2): the y-upwind entry is
    sqrt(1/2) = 0.707 of the x-upwind one, so the default threshold 0.99
    keeps only the x neighbour and the paper's 0.4 keeps both."""
    th = math.atan2(math.sqrt(1 / 3), math.sqrt(2 / 3))
    P = _grid(8, 8, th)
    assert abs(math.cos(th) - math.sqrt(2 / 3)) < 1e-15
    rid = P.A.row_ids()
    s = O.strength(P.A, 0.99)
    assert s.sum() == 64 - 15 and np.all(P.A.col[s] - rid[s] == -1)
    s4 = O.strength(P.A, 0.4)
    assert s4.sum() == 2 * (64 - 15)
    assert sorted(set((P.A.col[s4] - rid[s4]).tolist())) == [-8, -1]


def _path_graph(n):
    r = np.concatenate([np.arange(n - 1), np.arange(1, n)])
    c = np.concatenate([np.arange(1, n), np.arange(n - 1)])
    o = np.lexsort((c, r))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rowptr[1:])
    return rowptr, c[o].astype(np.int64)


def test_pmisr_hand_example_path():
    # path 0-1-2-3-4-5; degrees 1,2,2,2,2,1; weights decide among equal degrees
    rowptr, col = _path_graph(6)
    w = np.array([0, 10, 50, 20, 40, 0], dtype=np.uint32)
    is_f, rounds = O.pmisr(6, rowptr, col, w)
    # round 1: node 2 (deg 2, w 50) beats 1 and 3; node 4 (w 40) beats 3 and 5 -> F;
    # neighbours 1, 3, 5 -> C; node 0's only neighbour 1 is C -> round 2 makes 0 F.
    assert list(np.nonzero(is_f)[0]) == [0, 2, 4]
    assert rounds == 2


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pmisr_independent_and_maximal(seed):
    P = _grid(40, 30, 0.2 + seed)
    s = O.strength(P.A, 0.5)
    rp, gc = O.symmetrized_graph(P.A, s)
    is_f, _ = O.pmisr(P.A.n_rows, rp, gc, O.rng_u32(seed, 0, O.PURPOSE_PMISR, P.A.n_rows))
    src = np.repeat(np.arange(P.A.n_rows), np.diff(rp))
    assert not np.any(is_f[src] & is_f[gc])                  # F independent in S+S^T
    has_f_nb = np.zeros(P.A.n_rows, bool)
    has_f_nb[src[is_f[gc]]] = True
    assert np.all(has_f_nb[~is_f])                           # every C has an F neighbour
    # no large off-diagonal in A_ff: F-F entries are all weak
    rid = P.A.row_ids()
    ff = is_f[rid] & is_f[P.A.col] & (rid != P.A.col)
    assert not np.any(s[ff])


def test_symmetrized_graph_is_s_plus_st():
    P = _grid(9, 7, 0.9)
    s = O.strength(P.A, 0.6)
    rp, gc = O.symmetrized_graph(P.A, s)
    n = P.A.n_rows
    S = np.zeros((n, n), bool)
    S[P.A.row_ids()[s], P.A.col[s]] = True
    G = np.zeros((n, n), bool)
    G[np.repeat(np.arange(n), np.diff(rp)), gc] = True
    assert np.array_equal(G, S | S.T)


def test_ddc_converts_closest_to_target():
    # 100 F points with distinct ratios 0.01*i (diagonal 1, one F neighbour)
    n = 200
    rows, cols, vals = [], [], []
    for i in range(100):
        rows += [i, i]; cols += [i, 100 + i]; vals += [1.0, 0.0]
    for i in range(100, 200):
        rows += [i]; cols += [i]; vals += [1.0]
    A = O.csr_from_entries(n, n, np.array(rows), np.array(cols), np.array(vals))
    # give F row i the coupling 0.01*(i+1) to F point (i+1)%100 instead
    rows, cols, vals = [], [], []
    for i in range(100):
        j = (i + 1) % 100
        e = sorted([(i, 1.0), (j, -0.01 * (i + 1))])
        for c, v in e:
            rows.append(i); cols.append(c); vals.append(v)
    for i in range(100, 200):
        rows.append(i); cols.append(i); vals.append(1.0)
    A = O.csr_from_entries(n, n, np.array(rows), np.array(cols), np.array(vals))
    is_f = np.zeros(n, bool); is_f[:100] = True
    out, nconv = O.ddc_pass(A, is_f, 0.05)
    assert nconv == 5                                   # ceil(0.05 * 100)
    assert set(np.nonzero(is_f & ~out)[0]) == {95, 96, 97, 98, 99}  # least dominant
    # worst case of Sec. 2.1: all ratios equal -> the closest boundary converts none
    rows, cols, vals = [], [], []
    for i in range(100):
        j = (i + 1) % 100
        for c, v in sorted([(i, 1.0), (j, -0.5)]):
            rows.append(i); cols.append(c); vals.append(v)
    A2 = O.csr_from_entries(100, 100, np.array(rows), np.array(cols), np.array(vals))
    out2, n2 = O.ddc_pass(A2, np.ones(100, bool), 0.01)
    assert n2 == 0 and out2.all()


def test_ddc_ratio_definition():
    P = _grid(6, 6, 0.7)
    is_f = np.zeros(36, bool); is_f[::2] = True
    r = O.ddc_ratio(P.A, is_f)
    D = P.A.to_dense()
    for i in range(36):
        if is_f[i]:
            off = sum(abs(D[i, j]) for j in range(36) if j != i and is_f[j])
            assert r[i] == pytest.approx(off / abs(D[i, i]), rel=1e-15)
        else:
            assert r[i] == -1.0


def test_extract_blocks_reassemble():
    P = _grid(12, 9, 1.1)
    rng = np.random.default_rng(5)
    is_f = rng.random(P.A.n_rows) < 0.5
    D = P.A.to_dense()
    f, c = np.nonzero(is_f)[0], np.nonzero(~is_f)[0]
    assert np.array_equal(O.extract(P.A, is_f, is_f).to_dense(), D[np.ix_(f, f)])
    assert np.array_equal(O.extract(P.A, is_f, ~is_f).to_dense(), D[np.ix_(f, c)])
    assert np.array_equal(O.extract(P.A, ~is_f, is_f).to_dense(), D[np.ix_(c, f)])
    assert np.array_equal(O.extract(P.A, ~is_f, ~is_f).to_dense(), D[np.ix_(c, c)])


# ------------------------------------------------------ GMRES polynomials --
def _diag_dominant(n, seed):
    rng = np.random.default_rng(seed)
    D = np.diag(2.0 + rng.random(n))
    mask = rng.random((n, n)) < 0.15
    D = D + np.where(mask & ~np.eye(n, dtype=bool), rng.uniform(-0.3, 0.3, (n, n)), 0.0)
    r, c = np.nonzero(D)
    return O.csr_from_entries(n, n, r, c, D[r, c]), D


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_gmres_coeffs_equal_bruteforce_least_squares(p):
    """alpha minimises ||b - A q(A) b|| over degree-p polynomials (Eq. 7)."""
    A, D = _diag_dominant(40, p)
    opts = O.Options(poly_order=p)
    alpha, k, broke = O.gmres_poly_coeffs(A, opts, 3)
    assert k == p + 1 and not broke
    b = O.rng_uniform(opts.seed, 3, O.PURPOSE_COEF, 40)
    K = np.stack([np.linalg.matrix_power(D, j) @ b for j in range(p + 1)], axis=1)
    abf = np.linalg.lstsq(D @ K, b, rcond=None)[0]
    assert np.allclose(alpha, abf, rtol=1e-8, atol=1e-10)
    assert np.allclose(K @ alpha, K @ abf, rtol=1e-11, atol=1e-12)
    # Horner application equals the dense polynomial
    t = np.random.default_rng(9).standard_normal(40)
    qd = sum(alpha[j] * np.linalg.matrix_power(D, j) for j in range(p + 1))
    assert np.allclose(O.horner_apply(A, alpha, t), qd @ t, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_givens_least_squares_against_lapack(k):
    """The Givens solution of min ||beta e1 - H y|| for a (k+1) x k upper
    Hessenberg H, and its residual (the Arnoldi stopping test of reading 8),
    equal numpy's least-squares solution and residual."""
    rng = np.random.default_rng(40 + k)
    H = np.triu(rng.standard_normal((k + 1, k)), -1)
    beta = 0.5 + rng.random()
    e1 = np.zeros(k + 1)
    e1[0] = beta
    y_ref = np.linalg.lstsq(H, e1, rcond=None)[0]
    res_ref = np.linalg.norm(e1 - H @ y_ref)
    assert np.allclose(O.givens_lsq(H, beta), y_ref, rtol=1e-10, atol=1e-12)
    assert abs(O.givens_residual(H, beta) - res_ref) <= 1e-12 * max(res_ref, beta)


def test_gmres_coeffs_scaled_identity_breakdown():
    n, d = 30, 2.5
    A = O.csr_from_entries(n, n, np.arange(n), np.arange(n), np.full(n, d))
    alpha, k, broke = O.gmres_poly_coeffs(A, O.Options(poly_order=6), 0)
    assert broke and k == 1
    assert alpha[0] == pytest.approx(1.0 / d, rel=1e-15) and np.all(alpha[1:] == 0.0)


def test_fixed_sparsity_inverse_dense_check():
    A, D = _diag_dominant(25, 11)
    alpha = np.array([0.9, -0.4, 0.15, -0.05])
    Ah = O.fixed_sparsity_inverse(A, alpha)
    M = D != 0
    T = D.copy()
    acc = alpha[0] * np.eye(25) + alpha[1] * D
    for k in range(2, 4):
        T = np.where(M, D @ T, 0.0)
        acc = acc + alpha[k] * T
    assert np.allclose(Ah.to_dense(), np.where(M, acc, 0.0), rtol=1e-13, atol=1e-15)
    # a diagonal A_ff is closed under powers: the assembled inverse equals q(A)
    Dg = O.csr_from_entries(5, 5, np.arange(5), np.arange(5), np.arange(1.0, 6.0))
    Ahd = O.fixed_sparsity_inverse(Dg, alpha)
    x = np.arange(1.0, 6.0)
    assert np.allclose(Ahd.val, alpha[0] + alpha[1] * x + alpha[2] * x ** 2 + alpha[3] * x ** 3)


def test_restrictor_block_dense_check():
    A, D = _diag_dominant(30, 4)
    f = np.arange(30) % 3 != 0
    Aff = O.extract(A, f, f); Acf = O.extract(A, ~f, f)
    alpha = np.array([0.5, -0.1, 0.02])
    Ah = O.fixed_sparsity_inverse(Aff, alpha)
    Z = O.restrictor_block(Acf, Ah, 0.05)
    Zd = -(Acf.to_dense() @ Ah.to_dense())
    m = np.abs(Zd).max(1, keepdims=True)
    keep = (Zd != 0) & (np.abs(Zd) >= 0.05 * m)
    assert np.array_equal(Z.to_dense() != 0, keep)
    assert np.allclose(Z.to_dense(), np.where(keep, Zd, 0.0), rtol=1e-13, atol=1e-15)


def test_one_point_prolongator():
    P = _grid(10, 10, 3 * math.pi / 8)
    s = O.strength(P.A, 0.99)
    rp, gc = O.symmetrized_graph(P.A, s)
    is_f, _ = O.pmisr(100, rp, gc, O.rng_u32(1, 0, O.PURPOSE_PMISR, 100))
    W = O.one_point(P.A, s, is_f)
    c_ids = np.nonzero(~is_f)[0]
    D = P.A.to_dense()
    for fi, i in enumerate(np.nonzero(is_f)[0]):
        cands = [j for j in np.nonzero(D[i])[0] if j != i and not is_f[j]]
        if not cands:
            assert W[fi] == -1
            continue
        strongc = [j for j in cands if s[P.A.rowptr[i] + list(P.A.col[P.A.rowptr[i]:P.A.rowptr[i + 1]]).index(j)]]
        pool = strongc or cands
        best = max(pool, key=lambda j: (abs(D[i, j]), -j))
        assert c_ids[W[fi]] == best
    # P = [W; I] with weight 1 preserves constants on rows that have a C neighbour


def test_coarse_matrix_is_rap_and_lumping_keeps_row_sums():
    P = _grid(14, 14, 1.0)
    opts = O.Options(poly_order=3)
    strong, is_f, _, _ = O.cf_split(P.A, opts, 0)
    Aff = O.extract(P.A, is_f, is_f); Acf = O.extract(P.A, ~is_f, is_f)
    alpha, _, _ = O.gmres_poly_coeffs(Aff, opts, 0)
    Z = O.restrictor_block(Acf, O.fixed_sparsity_inverse(Aff, alpha), opts.r_drop)
    W = O.one_point(P.A, strong, is_f)
    n, nf = P.A.n_rows, int(is_f.sum())
    f, c = np.nonzero(is_f)[0], np.nonzero(~is_f)[0]
    R = np.zeros((n - nf, n)); R[:, f] = Z.to_dense(); R[np.arange(n - nf), c] = 1.0
    Pd = np.zeros((n, n - nf)); Pd[c, np.arange(n - nf)] = 1.0
    Pd[f[W >= 0], W[W >= 0]] = 1.0
    RAP = R @ P.A.to_dense() @ Pd
    Ac0 = O.coarse_matrix(P.A, is_f, Z, W, 0.0, True)         # no dropping
    assert np.allclose(Ac0.to_dense(), RAP, rtol=1e-12, atol=1e-14)
    Ac = O.coarse_matrix(P.A, is_f, Z, W, 0.3, True)          # heavy drop with lumping
    assert Ac.nnz < Ac0.nnz
    assert np.allclose(Ac.to_dense().sum(1), RAP.sum(1), rtol=1e-12, atol=1e-13)
    Acn = O.coarse_matrix(P.A, is_f, Z, W, 0.3, False)        # without lumping: diag unchanged
    assert np.array_equal(np.diag(Acn.to_dense()), np.diag(Ac0.to_dense()))


# ------------------------------------------------ coarse Newton polynomial --
def test_newton_polynomial_full_krylov_is_exact_inverse():
    A, D = _diag_dominant(24, 8)
    opts = O.Options()
    roots, H, k, broke = O.coarse_polynomial(A, opts, 0, 24)
    b = np.random.default_rng(2).standard_normal(24)
    x = O.newton_apply(A, roots, b)
    assert np.linalg.norm(b - D @ x) / np.linalg.norm(b) < 1e-10
    # harmonic Ritz values of the full Krylov space are the eigenvalues of A
    # (checked on a small matrix with a separated spectrum, where Arnoldi
    # keeps its basis orthogonal)
    n = 8
    Dm = np.diag(np.arange(1.0, n + 1)) + 0.05 * np.tril(np.ones((n, n)), -1)
    r, c = np.nonzero(Dm)
    Am = O.csr_from_entries(n, n, r, c, Dm[r, c])
    _, Hm, km, brm = O.coarse_polynomial(Am, opts, 0, n)
    th = np.sort_complex(O.harmonic_ritz(Hm, km, brm))
    assert km == n
    assert np.allclose(th, np.arange(1.0, n + 1), atol=1e-6)


def test_newton_form_equals_power_form():
    A, D = _diag_dominant(50, 13)
    opts = O.Options()
    b1 = O.rng_uniform(opts.seed, 0, O.PURPOSE_COARSE, 50)
    H, k, broke, beta = O.arnoldi(A, b1, 5, 1e-8)
    roots = O.order_roots(O.harmonic_ritz(H, k, broke), opts)
    alpha = O.power_coefficients(H, beta, O.givens_lsq(H, beta))
    v = np.random.default_rng(0).standard_normal(50)
    assert np.allclose(O.newton_apply(A, roots, v), O.horner_apply(A, alpha, v), rtol=1e-9, atol=1e-10)
    # residual polynomial prod(1 - z/theta) is 1 at z = 0 and q(A) b1 is the GMRES iterate
    x = O.newton_apply(A, roots, b1)
    K = np.stack([np.linalg.matrix_power(D, j) @ b1 for j in range(5)], 1)
    ybf = np.linalg.lstsq(D @ K, b1, rcond=None)[0]
    assert np.allclose(x, K @ ybf, rtol=1e-8)


@pytest.mark.parametrize("k", [3, 5, 7])
def test_harmonic_ritz_values_from_their_definition(k):
    """Harmonic Ritz values (Sec. 2.3) of A over K_k(A, b) are the theta with
    (A - theta I) y orthogonal to A K_k for some y in K_k.  With an
    orthonormal basis V of K_k (numpy QR of the monomial basis) and W = A V
    that is the generalised eigenproblem (W^T W) g = theta (W^T V) g, solved
    here by scipy: it must give the oracle's eig(H_k + h^2 H_k^-T e_k e_k^T)
    from its Arnoldi Hessenberg (k below n, so the h^2 term is present)."""
    sla = pytest.importorskip("scipy.linalg")
    n = 40
    A, D = _diag_dominant(n, 17 + k)
    b = O.rng_uniform(3, 0, O.PURPOSE_COARSE, n)
    H, kk, broke, _ = O.arnoldi(A, b, k, 1e-14, 0.0)
    assert kk == k and not broke and H[k, k - 1] > 1e-3
    K = np.stack([np.linalg.matrix_power(D, j) @ b for j in range(k)], 1)
    V, _ = np.linalg.qr(K)
    W = D @ V
    ref = np.sort_complex(sla.eigvals(W.T @ W, W.T @ V))
    got = np.sort_complex(O.harmonic_ritz(H, kk, broke))
    assert np.allclose(got, ref, rtol=1e-8, atol=1e-10)
    # and they differ from the plain Ritz values eig(H_k) when h_{k+1,k} != 0
    assert not np.allclose(np.sort_complex(np.linalg.eigvals(H[:k, :k])), ref, rtol=1e-6)


def test_leja_order_hand_examples():
    """Leja order (Sec. 2.3): the largest root first, then each next root
    maximises the product of distances to the roots already taken (both
    members of a taken pair count); a conjugate pair is one entry (im > 0).
    Worked by hand: {1, 2, 4, 8} -> 8 (largest); 1 (distance 7); 4 (4*3 = 12
    against 6*1 = 6 for 2); 2.  {3, 0.5, 1 +- i} -> 3; 0.5 (2.5 against
    |1 + i - 3| = 2.24); the pair."""
    opts = O.Options(addroot_log10=1e300)           # no added copies
    assert O.order_roots([1.0, 2.0, 4.0, 8.0], opts) == [(8.0, 0.0), (1.0, 0.0), (4.0, 0.0), (2.0, 0.0)]
    got = O.order_roots([1 + 1j, 0.5, 1 - 1j, 3.0], opts)
    assert got == [(3.0, 0.0), (0.5, 0.0), (1.0, 1.0)]
    # the added-copy reading: a root whose other factors |1 - z/theta_i|
    # multiply to 10^6 > 10^4 gets ceil((6 - 4) / 14) = 1 copy, appended
    opts = O.Options()
    assert (opts.addroot_log10, opts.addroot_per) == (4.0, 14.0)
    got = O.order_roots([1.0, 1000001.0], opts)
    assert got == [(1000001.0, 0.0), (1.0, 0.0), (1000001.0, 0.0)]


@pytest.mark.parametrize("roots", [[(2.0, 0.0), (1.5, 0.7), (3.0, 0.0)],
                                   [(2.5, 0.0), (1.2, 0.4)],
                                   [(1.7, 0.0)],
                                   [(0.9, 1.1), (2.2, 0.3)]])
def test_truncation_residual_is_residual_polynomial(roots):
    """Sec. 2.4 tests ||b2 - A q(A) b2|| / ||b2||.  For q in Newton form
    (Sec. 2.3), b2 - A q(A) b2 = prod_i (I - A / theta_i) b2 over every root,
    a pair a +- ib contributing both conjugates: the product is formed
    densely in complex arithmetic, for real roots and pairs in any position
    (the last one included)."""
    n, level = 30, 3
    A, D = _diag_dominant(n, 5)
    opts = O.Options()
    R = np.eye(n, dtype=complex)
    for a, bi in roots:
        for th in ([complex(a, 0.0)] if bi == 0.0 else [complex(a, bi), complex(a, -bi)]):
            R = R @ (np.eye(n) - D / th)
    b2 = O.rng_uniform(opts.seed, level, O.PURPOSE_TRUNC, n)
    rb = R @ b2
    assert np.max(np.abs(rb.imag)) < 1e-12 * np.max(np.abs(rb.real))
    expected = np.linalg.norm(rb.real) / np.linalg.norm(b2)
    got = O.truncation_residual(A, roots, opts, level)
    assert abs(got - expected) <= 1e-12 * expected


# ------------------------------------------------------------- V-cycle ----
def test_grid_aligned_direction_is_exact_solver():
    """v = (1, 0): uncoupled 1D chains; A_ff diagonal, ideal R, exact
    F-smoothing: the V-cycle is an exact inverse (Sec. 2 and 3.4)."""
    P = O.advection_2d(32, 24, 1.0, 0.0)
    opts = O.Options(trunc_rtol=0.0, coarse_min_rows=40)
    H = O.setup(P.A, opts)
    assert len(H.levels) >= 2
    for L in H.levels:
        assert np.all(L.A_ff.col == L.A_ff.row_ids())          # diagonal A_ff
    r = np.random.default_rng(1).standard_normal(P.A.n_rows)
    e = O.vcycle(H, r)
    assert np.linalg.norm(r - P.A.to_dense() @ e) / np.linalg.norm(r) < 1e-12
    b = O.assemble_rhs(P, np.random.default_rng(2).random(P.inflow.size), np.zeros(P.A.n_rows))
    x, info = O.solve(H, P.A, b)
    assert info.iterations <= 2 and info.converged


def test_c1_constant_solution_and_convergence():
    P = _grid(64, 64, 3 * math.pi / 8)
    b = O.assemble_rhs(P, np.ones(P.inflow.size), np.zeros(4096))
    H = O.setup(P.A, O.Options(poly_order=4, trunc_start_level=4))
    assert len(H.levels) >= 3
    x, info = O.solve(H, P.A, b, rtol=1e-10)
    assert info.converged
    assert np.linalg.norm(b - P.A.to_dense() @ x) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x - 1.0) / np.linalg.norm(np.ones(4096)) < 1e-9
    assert info.iterations <= 12


def test_solution_matches_sweep_random_inflow_and_source():
    P = _grid(48, 40, 0.9)
    rng = np.random.default_rng(4)
    b = O.assemble_rhs(P, rng.random(P.inflow.size), rng.standard_normal(P.A.n_rows))
    H = O.setup(P.A, O.Options(trunc_start_level=1))
    x, info = O.solve(H, P.A, b, rtol=1e-12)
    u = O.sweep_solve(P.A, b, O.sweep_order(P))
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-9


def test_truncation_reduces_levels():
    P = _grid(64, 64, math.pi / 4)
    full = O.setup(P.A, O.Options(trunc_rtol=0.0, coarse_min_rows=8))
    trunc = O.setup(P.A, O.Options(trunc_rtol=0.1, coarse_poly_order=30, trunc_start_level=1))
    assert trunc.truncated and len(trunc.levels) < len(full.levels)
    assert trunc.coarse_trunc_rel <= 0.1
    for L in trunc.levels[1:]:
        assert L.trunc_rel > 0.1                     # levels kept had failed the test


def test_complexities_in_paper_range():
    """Sanity band (not parity): pi/4, order 6 smoother (Sec. 3)."""
    P = _grid(128, 128, math.pi / 4)
    H = O.setup(P.A, O.Options(trunc_rtol=0.0, coarse_min_rows=16))
    cx = O.complexities(H)
    assert 10 < cx["cycle"] < 60
    assert 2 < cx["storage"] < 20


@pytest.mark.parametrize("opts", [dict(), dict(smoother="assembled"), dict(smooth_type="fc"),
                                  dict(smooth_type="fcf", smoother="assembled"), dict(poly_order=0)])
def test_complexities_count_what_one_vcycle_does(opts, monkeypatch):
    """Sec. 3 defines the cycle complexity as the FLOPs of one V-cycle over
    those of one top-level SpMV, and the storage complexity as the non-zeros
    of every matrix the solve needs over nnz(A_top).  Every SpMV of the
    oracle's V-cycle is counted here as it runs (2 flops per stored entry),
    and the distinct matrices it touches are collected; the top matrix (the
    outer residual), R's identity block (n_c) and the one-point P (one index
    per F row plus its identity block) complete the storage.  The coarse
    polynomial of this case has real roots and conjugate pairs."""
    P = _grid(48, 40, 0.9)
    H = O.setup(P.A, O.Options(trunc_start_level=1, **opts))
    assert any(im > 0 for _, im in H.roots) and any(im == 0 for _, im in H.roots)
    flops, mats = [0], {}
    real_spmv = O.spmv

    def counting_spmv(A, x):
        flops[0] += 2 * A.nnz
        mats[id(A)] = A.nnz
        return real_spmv(A, x)

    monkeypatch.setattr(O, "spmv", counting_spmv)
    O.vcycle(H, np.random.default_rng(1).standard_normal(P.A.n_rows))
    monkeypatch.setattr(O, "spmv", real_spmv)
    top = P.A.nnz
    cx = O.complexities(H)
    assert cx["cycle"] == flops[0] / (2.0 * top)
    blocks = sum(2 * int((~L.is_f).sum()) + int(L.is_f.sum()) for L in H.levels)
    assert cx["storage"] == (top + sum(mats.values()) + blocks) / top


def test_dense_adjoint():
    P = _grid(12, 12, 0.5)
    rhs = np.random.default_rng(0).standard_normal(144)
    lam = O.dense_adjoint(P.A, rhs)
    assert np.allclose(P.A.to_dense().T @ lam, rhs, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_fgmres_iterate_minimises_residual_over_its_space(k):
    """With a fixed linear preconditioner M^-1 (one V-cycle), k steps of
    right-preconditioned (flexible) GMRES from x0 = 0 give the x in
    M^-1 K_k(A M^-1, b) with the smallest ||b - A x||_2: formed here from
    dense M^-1 (the V-cycle applied to the unit vectors), a monomial Krylov
    basis and numpy least squares.  The recorded residual history equals
    the true residual of that iterate."""
    P = _grid(13, 11, 0.7)
    n = P.A.n_rows
    H = O.setup(P.A, O.Options(poly_order=2, trunc_start_level=1))
    b = O.assemble_rhs(P, np.random.default_rng(9).random(P.inflow.size),
                       np.random.default_rng(10).standard_normal(n))
    Minv = np.stack([O.vcycle(H, e) for e in np.eye(n)], 1)
    A = P.A.to_dense()
    B = A @ Minv
    K = np.stack([np.linalg.matrix_power(B, j) @ b for j in range(k)], 1)
    y = np.linalg.lstsq(B @ K, b, rcond=None)[0]
    x_ref = Minv @ (K @ y)
    x, info = O.fgmres(P.A, b, lambda r: O.vcycle(H, r), rtol=0.0, restart=30, maxit=k)
    assert info.iterations == k
    nb = np.linalg.norm(b)
    assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    assert abs(info.history[k] - np.linalg.norm(b - A @ x) / nb) <= 1e-10


def test_richardson_iterates_match_closed_form():
    """The V-cycle is a fixed linear map B (fixed polynomials, fixed
    operators), so Richardson from x0 = 0 gives the partial Neumann sums
    x_k = sum_{i<k} (I - B A)^i B b exactly; B is formed column by column."""
    P = _grid(12, 10, 0.7)
    n = P.A.n_rows
    H = O.setup(P.A, O.Options(poly_order=3, trunc_start_level=1))
    Bm = np.column_stack([O.vcycle(H, np.eye(n)[:, i]) for i in range(n)])
    Ad = P.A.to_dense()
    b = np.random.default_rng(11).standard_normal(n)
    x, info = O.richardson(P.A, b, lambda v: O.vcycle(H, v), rtol=0.0, atol=0.0, maxit=3)
    E = np.eye(n) - Bm @ Ad
    ref = Bm @ b + E @ (Bm @ b) + E @ (E @ (Bm @ b))
    assert info.iterations == 3
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-12


def test_richardson_exact_preconditioner_and_sweep():
    """Grid-aligned flow: the V-cycle is exact, one Richardson step solves.
    Skewed flow: Richardson reaches the sweep solution."""
    P = O.advection_2d(32, 24, 1.0, 0.0)
    H = O.setup(P.A, O.Options(trunc_rtol=0.0, coarse_min_rows=40))
    b = O.assemble_rhs(P, np.random.default_rng(2).random(P.inflow.size), np.zeros(P.A.n_rows))
    x, info = O.solve(H, P.A, b, rtol=1e-11, outer="richardson")
    assert info.iterations == 1 and info.converged
    P = _grid(48, 40, 0.9)
    rng = np.random.default_rng(4)
    b = O.assemble_rhs(P, rng.random(P.inflow.size), rng.standard_normal(P.A.n_rows))
    H = O.setup(P.A, O.Options(trunc_start_level=1))
    x, info = O.solve(H, P.A, b, rtol=1e-12, outer="richardson")
    u = O.sweep_solve(P.A, b, O.sweep_order(P))
    assert info.converged
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-9


def test_assembled_smoother_equals_polynomial_at_degree_one():
    """At smoother degree 1, q(A_ff) = a0 I + a1 A_ff is its own
    fixed-sparsity matrix (Eq. 8 has no masked power), so the V-cycle with the
    assembled inverse equals the matrix-free one up to rounding; a wrong
    stored inverse or a wrong application breaks this."""
    P = _grid(40, 36, 1.1)
    hp = O.setup(P.A, O.Options(poly_order=1, trunc_start_level=1))
    ha = O.setup(P.A, O.Options(poly_order=1, trunc_start_level=1, smoother="assembled"))
    r = np.random.default_rng(5).standard_normal(P.A.n_rows)
    ep, ea = O.vcycle(hp, r), O.vcycle(ha, r)
    assert np.linalg.norm(ep - ea) <= 1e-13 * np.linalg.norm(ep)
    # at degree 6 the masked powers make them differ
    hp6 = O.setup(P.A, O.Options(trunc_start_level=1))
    ha6 = O.setup(P.A, O.Options(trunc_start_level=1, smoother="assembled"))
    assert np.linalg.norm(O.vcycle(hp6, r) - O.vcycle(ha6, r)) > 1e-8 * np.linalg.norm(ep)


def test_assembled_smoother_exact_and_convergent():
    """Grid-aligned flow: A_ff = d I, the stored inverse is exact and one
    iteration solves.  Skewed flow: converges to the sweep solution; the
    storage complexity grows by the stored inverses."""
    P = O.advection_2d(32, 24, 1.0, 0.0)
    H = O.setup(P.A, O.Options(trunc_rtol=0.0, coarse_min_rows=40, smoother="assembled"))
    b = O.assemble_rhs(P, np.random.default_rng(2).random(P.inflow.size), np.zeros(P.A.n_rows))
    x, info = O.solve(H, P.A, b, rtol=1e-11)
    assert info.iterations <= 1 and info.converged
    P = _grid(48, 40, 0.9)
    rng = np.random.default_rng(4)
    b = O.assemble_rhs(P, rng.random(P.inflow.size), rng.standard_normal(P.A.n_rows))
    ha = O.setup(P.A, O.Options(trunc_start_level=1, smoother="assembled"))
    hp = O.setup(P.A, O.Options(trunc_start_level=1))
    x, info = O.solve(ha, P.A, b, rtol=1e-12)
    u = O.sweep_solve(P.A, b, O.sweep_order(P))
    assert info.converged and np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-9
    ca, cp = O.complexities(ha), O.complexities(hp)
    extra = sum(L.Ainv.nnz for L in ha.levels) / P.A.nnz
    assert abs(ca["storage"] - cp["storage"] - extra) < 1e-12


@pytest.mark.parametrize("theta", [0.5, 1.0, 3.5])
def test_c_point_smoothing_zeroes_its_block_residual(theta):
    """Block smoothing with an exact block inverse zeroes that block's
    residual (Sec. 2, Eq. 6 and its C-point analogue): on a 7 x 6 grid every
    level is small enough that the GMRES polynomials of A_ff and A_cc reach
    the exact inverse (the Krylov space breaks down), and the coarse
    polynomial is exact.  After one V-cycle from zero, the residual r - A e
    is zero on the F points when the last smooth is an F-point smooth (f,
    fcf) and zero on the C points after an fc cycle; the other block's
    residual is not (the check is not vacuous)."""
    P = _grid(7, 6, theta)
    r = np.random.default_rng(0).standard_normal(P.A.n_rows)
    res = {}
    for st in ("f", "fc", "fcf"):
        H = O.setup(P.A, O.Options(poly_order=45, coarse_poly_order=100, trunc_rtol=0.0, smooth_type=st))
        L = H.levels[0]
        assert L.alpha_k <= L.A_ff.n_rows and (st == "f" or L.alpha_c_k <= L.A_cc.n_rows)
        e = O.vcycle(H, r)
        rr = r - O.spmv(P.A, e)
        res[st] = (np.linalg.norm(rr[L.is_f]), np.linalg.norm(rr[~L.is_f]))
    nr = np.linalg.norm(r)
    assert res["f"][0] <= 1e-12 * nr and res["f"][1] > 1e-3 * nr
    assert res["fc"][1] <= 1e-12 * nr and res["fc"][0] > 1e-3 * nr
    assert res["fcf"][0] <= 1e-12 * nr and res["fcf"][1] > 1e-4 * nr


def test_c_point_smoothing_storage_is_the_rest_of_a():
    """C-point smoothing keeps A_cf and A_cc, so per level the stored blocks
    add up to all of A_l (the four blocks of Eq. 3 partition A)."""
    P = _grid(40, 36, 0.9)
    Hf = O.setup(P.A, O.Options(smooth_type="f"))
    Hc = O.setup(P.A, O.Options(smooth_type="fc"))
    top = P.A.nnz
    extra = sum(L.A.nnz - L.A_ff.nnz - L.A_fc.nnz for L in Hc.levels)
    sf, sc = O.complexities(Hf)["storage"], O.complexities(Hc)["storage"]
    assert abs((sc - sf) * top - extra) < 1e-6
    for L in Hc.levels:
        assert L.A_cf.nnz + L.A_cc.nnz + L.A_ff.nnz + L.A_fc.nnz == L.A.nnz


def _neumann_q(A, p):
    """Dense q(A) from the oracle's power-basis Neumann coefficients."""
    al = O.neumann_coeffs(A, O.Options(poly_order=p))
    D = A.to_dense()
    Q = np.zeros_like(D)
    Pk = np.eye(D.shape[0])
    for a in al:
        Q += a * Pk
        Pk = Pk @ D
    return al, D, Q


@pytest.mark.parametrize("p", [0, 1, 4, 6])
def test_neumann_residual_polynomial(p):
    """The truncated Neumann series fixes its own residual: with w = 1 / max
    |a_ii|, I - A q(A) = (I - w A)^(p+1) (Sec. 3.3.1 nAIR; the identity of a
    geometric sum).  Checked on the A_ff of a real level, whose diagonal is
    the constant |vx| + |vy|."""
    P = _grid(12, 10, 0.7)
    H = O.setup(P.A, O.Options(max_levels=2, trunc_rtol=0.0))
    A_ff = H.levels[0].A_ff
    al, D, Q = _neumann_q(A_ff, p)
    w = 1.0 / np.max(np.abs(np.diag(D)))
    assert abs(w - 1.0 / (math.cos(0.7) + math.sin(0.7))) < 1e-15
    E = np.linalg.matrix_power(np.eye(D.shape[0]) - w * D, p + 1)
    assert np.max(np.abs(np.eye(D.shape[0]) - D @ Q - E)) < 1e-13


def test_neumann_exact_on_nilpotent_part():
    """A = d (I - N) with N strictly lower bidiagonal (nilpotent, N^n = 0):
    the series of degree n - 1 is the exact inverse; A = d I gives q = 1/d
    at every degree."""
    n, d = 6, 1.7
    rows = list(range(n)) + list(range(1, n))
    cols = list(range(n)) + list(range(n - 1))
    vals = [d] * n + [-0.9] * (n - 1)
    o = np.lexsort((cols, rows))
    A = O.csr_from_entries(n, n, np.array(rows)[o], np.array(cols)[o], np.array(vals)[o])
    _, D, Q = _neumann_q(A, n - 1)
    assert np.max(np.abs(Q - np.linalg.inv(D))) < 1e-12
    I = O.csr_from_entries(4, 4, np.arange(4), np.arange(4), np.full(4, d))
    for p in (0, 3):
        _, _, Qi = _neumann_q(I, p)
        assert np.max(np.abs(Qi - np.eye(4) / d)) < 1e-15


def test_nair_solves_the_constant_inflow_problem():
    """nAIR (Neumann smoother and Neumann-based Z) on the 64 x 64 problem with
    g = 1, s = 0 converges to the closed-form u = 1 (Eq. 1-2)."""
    P = _grid(64, 64, 3 * math.pi / 8)
    b = O.assemble_rhs(P, np.ones(P.inflow.size), np.zeros(P.A.n_rows))
    H = O.setup(P.A, O.Options(poly_order=4, inverse_type="neumann", trunc_start_level=4))
    x, info = O.solve(H, P.A, b, rtol=1e-10)
    assert info.converged and np.max(np.abs(x - 1.0)) < 1e-8
    assert H.levels[0].alpha_k == 5


@pytest.mark.parametrize("st", ["fc", "fcf"])
def test_assembled_c_point_smoothing_equals_matrix_free_at_degree_one(st):
    """At degree p = 1 the polynomial a_0 I + a_1 A already has the pattern
    of A plus the diagonal, so the fixed-sparsity inverse of Eq. 8 is the
    polynomial itself.  The assembled F- and C-point smoothers must then
    give the same V-cycle as the matrix-free ones (pinned by block
    exactness above), for FC and FCF alike."""
    P = _grid(30, 26, 1.1)
    r = np.random.default_rng(2).standard_normal(P.A.n_rows)
    out = {}
    for sm in ("polynomial", "assembled"):
        H = O.setup(P.A, O.Options(poly_order=1, coarse_poly_order=30, trunc_rtol=1e-2, smooth_type=st,
                                   smoother=sm))
        out[sm] = O.vcycle(H, r)
        if sm == "assembled":
            assert all(L.Ainv_cc is not None for L in H.levels)
    assert np.linalg.norm(out["assembled"] - out["polynomial"]) <= 1e-13 * np.linalg.norm(out["polynomial"])
