"""CPU-only checks of the CUDA library: it loads, exports every entry point
declared in include/airg.h, and its host-side FP64 steps agree with the
oracle (no GPU calls)."""
import os
import re

import numpy as np
import pytest

import paper_2508_17517_gb300 as G
from oracle import airg as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    G.build()
    return G.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "airg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(airg_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_binding_names():
    assert _declared() == sorted(G.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_binding_argument_types_match_header_prototypes(L):
    """Every ctypes signature of the binding agrees with its prototype in
    include/airg.h: same number of arguments, pointers where the header has
    pointers, and scalars of the same width and kind (integer or floating)."""
    import ctypes
    txt = open(os.path.join(ROOT, "include", "airg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = re.findall(r"\b(airg_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", txt)
    assert sorted(n for n, _ in protos) == _declared()
    scalars = {"int": ctypes.c_int, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
               "uint64_t": ctypes.c_uint64, "double": ctypes.c_double, "float": ctypes.c_float}
    floating = (ctypes.c_double, ctypes.c_float)
    for name, args in protos:
        args = [a.strip() for a in args.split(",") if a.strip() not in ("", "void")]
        at = getattr(L, name).argtypes
        assert at is not None and len(at) == len(args), name
        for a, t in zip(args, at):
            decl = re.sub(r"\bconst\b", "", a).split()
            if "*" in a:
                assert t is ctypes.c_void_p or issubclass(t, ctypes._Pointer), (name, a, t)
            elif decl[0] in scalars:
                e = scalars[decl[0]]
                assert ctypes.sizeof(t) == ctypes.sizeof(e) and (t in floating) == (e in floating), (name, a, t)


def test_options_default_are_paper_values(L):
    o = G.airg_options_default()
    assert (o.strong_threshold, o.ddc_fraction, o.ddc_its, o.poly_order) == (0.99, 0.01, 2, 6)
    assert (o.coarse_poly_order, o.trunc_rtol, o.a_drop, o.a_lump) == (100, 0.1, 1e-6, 1)
    d = O.Options()
    assert (o.r_drop, o.seed, o.breakdown_tol, o.exact_tol) == (d.r_drop, d.seed, d.breakdown_tol, d.exact_tol)


@pytest.mark.parametrize("seed", range(6))
def test_host_gmres_coeffs_bitwise_equal_to_oracle(L, seed):
    """The host least-squares + recurrence performs the same IEEE operations
    as the oracle, so the coefficients agree bit for bit."""
    rng = np.random.default_rng(seed)
    k = [1, 2, 3, 5, 7, 7][seed]
    if seed < 4:
        H = np.triu(rng.standard_normal((k + 1, k)), -1)
        H[np.arange(1, k + 1), np.arange(k)] = np.abs(H[np.arange(1, k + 1), np.arange(k)]) + 0.1
        beta = float(rng.random() + 0.5)
    else:
        A, _ = _dd(40, seed)
        b = O.rng_uniform(seed, 0, O.PURPOSE_COEF, 40)
        H, k2, broke, beta = O.arnoldi(A, b, k, 1e-8)
        assert k2 == k
    y = O.givens_lsq(H, beta)
    ref = np.array(O.power_coefficients(H, beta, y))
    got = G.airg_host_gmres_coeffs(H, beta)
    assert np.array_equal(got, ref)


def _dd(n, seed):
    rng = np.random.default_rng(seed)
    D = np.diag(2.0 + rng.random(n))
    D = D + np.where((rng.random((n, n)) < 0.15) & ~np.eye(n, dtype=bool), rng.uniform(-0.3, 0.3, (n, n)), 0)
    r, c = np.nonzero(D)
    return O.csr_from_entries(n, n, r, c, D[r, c]), D


@pytest.mark.parametrize("n", [1, 2, 3, 6, 17, 40, 100])
def test_host_eigvals_match_lapack(L, n):
    rng = np.random.default_rng(n)
    H = np.triu(rng.standard_normal((n, n)), -1)
    got = np.sort_complex(G.airg_host_eigvals(H))
    ref = np.sort_complex(np.linalg.eigvals(H))
    assert np.allclose(got, ref, rtol=1e-8, atol=1e-9 * max(1.0, np.abs(ref).max()))


def test_host_eigvals_of_arnoldi_hessenberg(L):
    A, D = _dd(60, 3)
    b = O.rng_uniform(1, 0, O.PURPOSE_COARSE, 60)
    H, k, broke, beta = O.arnoldi(A, b, 20, 1e-8)
    got = np.sort_complex(G.airg_host_eigvals(H[:k, :k]))
    ref = np.sort_complex(np.linalg.eigvals(H[:k, :k]))
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-10)


def test_host_argument_checks_need_no_gpu(L):
    """Invalid calls are rejected by host-side checks, before any CUDA call,
    with the documented status (AIRG_ERR_ARG = 1, AIRG_ERR_STATE = 7) and a
    message; nothing here reaches the device, so it runs without a GPU."""
    import ctypes
    ARG, STATE = 1, 7
    fake = ctypes.c_void_p(64)          # never dereferenced: every call fails first
    i64 = ctypes.c_int64()

    def err():
        return L.airg_last_error().decode()

    assert L.airg_options_default(None) == ARG and "null options" in err()
    h = ctypes.c_void_p()
    assert L.airg_setup(None, None, None, None) == ARG and "output handle" in err()
    assert L.airg_setup(None, None, None, ctypes.byref(h)) == ARG and "null CSR" in err()
    assert h.value is None
    for field, value, msg in [("poly_order", 31, "poly_order"), ("coarse_poly_order", 0, "coarse_poly_order"),
                              ("gmres_restart", 31, "gmres_restart"), ("precision", 9, "precision"),
                              ("smooth_type", 5, "smooth_type"), ("ddc_fraction", 1.5, "DDC")]:
        o = G.airg_options()
        L.airg_options_default(ctypes.byref(o))
        setattr(o, field, value)
        csr = G.airg_csr(4, 4, 4, fake, fake, fake, 0)
        assert L.airg_setup(ctypes.byref(csr), ctypes.byref(o), None, ctypes.byref(h)) == ARG, field
        assert msg in err(), (field, err())
    for n_rows, n_cols, nnz, msg in [(4, 5, 4, "square"), (0, 0, 0, "square"), (1 << 31, 1 << 31, 4, "2^31"),
                                     (4, 4, -1, "2^31")]:
        csr = G.airg_csr(n_rows, n_cols, nnz, fake, fake, fake, 0)
        assert L.airg_setup(ctypes.byref(csr), None, None, ctypes.byref(h)) == ARG and msg in err()
    assert L.airg_solve(None, 1, fake, fake, 1, 1e-10, 0.0, 10, None, None) == STATE
    assert L.airg_solve_adjoint(None, 1, fake, fake, 1, 1e-10, 0.0, 10, None, None) == STATE
    assert L.airg_setup_info(None, None) == ARG
    assert L.airg_export_matrix(None, 0, 0, ctypes.byref(i64), ctypes.byref(i64), ctypes.byref(i64),
                                None, None, None) == STATE
    assert L.airg_export_vector(None, 0, 0, ctypes.byref(i64), None) == STATE
    assert L.airg_profile(None, 1) == STATE
    one = G.airg_csr(4, 4, 4, fake, fake, fake, 0)
    assert L.airg_setup_batch(0, ctypes.byref(one), None, None, ctypes.byref(h)) == ARG
    assert L.airg_setup_batch(1, None, None, None, ctypes.byref(h)) == ARG
    assert L.airg_solve_batch(None, fake, fake, 1, 1e-10, 0.0, 10, None, None) == ARG
    assert L.airg_batch_setup_info(None, 0, None) == ARG
    assert L.airg_problem_advection2d(1, 8, 1.0, 0.0, 0.1, fake, fake, fake, fake, ctypes.byref(i64),
                                      ctypes.byref(i64), None) == ARG
    assert L.airg_problem_advection2d(8, 8, float("nan"), 0.0, 0.1, fake, fake, fake, fake,
                                      ctypes.byref(i64), ctypes.byref(i64), None) == ARG
    for bad_h in (-0.1, float("nan"), float("inf")):
        assert L.airg_problem_advection2d(8, 8, 1.0, 0.0, bad_h, fake, fake, fake, fake,
                                          ctypes.byref(i64), ctypes.byref(i64), None) == ARG
        assert L.airg_assemble_rhs_advection2d(8, 8, 1.0, 0.0, bad_h, 1, fake, 8, fake, None, fake, None) == ARG
        assert L.airg_rhs_adjoint_advection2d(8, 8, 1.0, 0.0, bad_h, 1, fake, 8, fake, fake, None, None) == ARG
    assert L.airg_assemble_rhs_advection2d(8, 8, 1.0, 0.0, 0.1, 0, fake, 8, fake, None, fake, None) == ARG
    assert L.airg_rhs_adjoint_advection2d(8, 8, 1.0, 0.0, 0.1, 1, fake, -1, fake, fake, None, None) == ARG
    assert L.airg_dot_exact_noalloc(-1, fake, fake, fake, None) == ARG
    assert L.airg_dot_exact_noalloc(1 << 31, fake, fake, fake, None) == ARG and "2^31" in err()
    d = ctypes.c_double()
    assert L.airg_dot_exact(-1, fake, fake, ctypes.byref(d), None) == ARG
    assert L.airg_dot_exact(1 << 31, fake, fake, ctypes.byref(d), None) == ARG and "2^31" in err()
    assert L.airg_check_wait_timeout(0, None) == ARG
    lay = G.airg_operator_layout()
    assert L.airg_operator_layout_info(None, 0, 0, ctypes.byref(lay)) == ARG and "null handle" in err()
    L.airg_free(None)
    L.airg_batch_free(None)


def test_header_is_plain_c_and_links_from_c(L, tmp_path):
    """include/airg.h compiles as strict C99 and a C program links against
    the library and calls it (defaults and a host-side argument check; no
    GPU call)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    src = tmp_path / "use_airg.c"
    src.write_text(
        '#include <stdio.h>\n#include "airg.h"\n'
        "int main(void) {\n"
        "  airg_options o;\n"
        "  airg_handle* h = 0;\n"
        "  if (airg_options_default(&o) != AIRG_OK) return 1;\n"
        "  o.poly_order = 99;\n"
        "  if (airg_setup(0, &o, 0, &h) != AIRG_ERR_ARG || h) return 2;\n"
        '  printf("%d %d %.2f %s\\n", o.ddc_its, o.coarse_poly_order, o.strong_threshold, airg_last_error());\n'
        '  printf("%d %d\\n", (int)sizeof(airg_operator_layout), (int)sizeof(airg_hierarchy_info));\n'
        "  airg_free(h);\n"
        "  return 0;\n"
        "}\n")
    libdir = os.path.dirname(G.LIB)
    exe = tmp_path / "use_airg"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lairg",
                        "-Wl,-rpath," + libdir, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.split()[:3] == ["2", "100", "0.99"] and "poly_order" in r.stdout
    # the binding's structs have the C layout's size
    import ctypes
    sizes = [int(v) for v in r.stdout.splitlines()[-1].split()]
    assert sizes == [ctypes.sizeof(G.airg_operator_layout), ctypes.sizeof(G.airg_hierarchy_info)]
