"""GB300 (sm_103a) AIRG: reduction multigrid with GMRES polynomials for advection.

Python binding of the C ABI declared in ``include/airg.h``: argument
marshalling only.  Every step of setup and solve runs in the CUDA library
``_lib/libairg.so`` (built by ``paper_2508_17517_gb300._build.build()``); if
that library is missing, the binding raises -- there is no CPU fallback.
Tensors are torch CUDA tensors; the current torch stream is passed to every
call.
"""
import ctypes
import os

import numpy as np

from ._build import LIB, build  # noqa: F401

AIRG_OK = 0
AIRG_ERR_NOT_CONVERGED = 5
AIRG_SMOOTH_POLYNOMIAL = 0
AIRG_SMOOTH_ASSEMBLED = 1
AIRG_SMOOTH_F = 0
AIRG_SMOOTH_FC = 1
AIRG_SMOOTH_FCF = 2
AIRG_INVERSE_GMRES = 0
AIRG_INVERSE_NEUMANN = 1
AIRG_OUTER_FGMRES = 0
AIRG_OUTER_RICHARDSON = 1
AIRG_FP64 = 0
AIRG_MIXED_FP32 = 1
AIRG_MIXED_FP32_BF16R = 2
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_BREAKDOWN",
                5: "ERR_NOT_CONVERGED", 6: "ERR_TIMEOUT", 7: "ERR_STATE"}

# symbols declared in include/airg.h
EXPORTS = ["airg_options_default", "airg_problem_advection2d", "airg_assemble_rhs_advection2d",
           "airg_setup", "airg_solve", "airg_solve_adjoint", "airg_setup_info",
           "airg_export_matrix", "airg_export_vector", "airg_free", "airg_last_error",
           "airg_dot_exact", "airg_rng_uniform", "airg_host_gmres_coeffs", "airg_host_eigvals",
           "airg_profile", "airg_profile_read", "airg_profile_read_level", "airg_dot_exact_noalloc",
           "airg_rhs_adjoint_advection2d", "airg_setup_batch", "airg_solve_batch",
           "airg_batch_free", "airg_batch_setup_info", "airg_check_wait_timeout", "airg_profile_group",
           "airg_batch_profile", "airg_batch_profile_read", "airg_operator_layout_info"]
PROFILE_KINDS = ["restrict", "f_residual", "f_smoother", "coarse_newton", "top_spmv",
                 "krylov_vectors", "layout"]
# airg_hierarchy_info.setup_phase_ms entries (AIRG_PHASE_* of the header)
SETUP_PHASES = ["truncation_test", "cf_split", "extract", "smoother_poly", "fixed_sparsity_inverse",
                "restrictor", "prolongator", "rap", "drop_lump", "coarse_poly", "solve_layout"]


class airg_options(ctypes.Structure):
    _fields_ = [("strong_threshold", ctypes.c_double), ("ddc_fraction", ctypes.c_double),
                ("ddc_its", ctypes.c_int), ("poly_order", ctypes.c_int),
                ("coarse_poly_order", ctypes.c_int), ("trunc_rtol", ctypes.c_double),
                ("trunc_start_level", ctypes.c_int), ("max_levels", ctypes.c_int),
                ("coarse_min_rows", ctypes.c_int), ("a_drop", ctypes.c_double),
                ("a_lump", ctypes.c_int), ("r_drop", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("breakdown_tol", ctypes.c_double), ("exact_tol", ctypes.c_double),
                ("addroot_log10", ctypes.c_double),
                ("addroot_per", ctypes.c_double), ("precision", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("outer", ctypes.c_int), ("smoother", ctypes.c_int),
                ("smooth_type", ctypes.c_int), ("inverse_type", ctypes.c_int)]


class airg_csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("on_device", ctypes.c_int)]


class airg_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("converged", ctypes.c_int), ("solve_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64)]


class airg_hierarchy_info(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("truncated", ctypes.c_int),
                ("coarse_roots", ctypes.c_int), ("coarse_krylov", ctypes.c_int),
                ("cycle_complexity", ctypes.c_double),
                ("storage_complexity", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("n", ctypes.c_int64 * 64), ("n_f", ctypes.c_int64 * 64),
                ("nnz_a", ctypes.c_int64 * 64), ("bytes_per_vcycle", ctypes.c_int64),
                ("setup_phase_ms", ctypes.c_double * 16), ("exact_dots", ctypes.c_int64)]


class airg_operator_layout(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("padded", ctypes.c_int64), ("warps_per_slice", ctypes.c_int32), ("r", ctypes.c_int32),
                ("resident_grid", ctypes.c_int32), ("index_bytes", ctypes.c_int32),
                ("slice_bases", ctypes.c_int32), ("value_bytes", ctypes.c_int32),
                ("dense_diagonal", ctypes.c_int32)]


# operators of airg_operator_layout_info (AIRG_OPERATOR_* of the header)
OPERATORS = ["top", "Z", "M", "A_ff", "Ainv", "C_rows", "A_cc", "Ainv_cc", "F_rows", "coarse"]


class AirgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("AIRG CUDA library not built (%s); run "
                               "paper_2508_17517_gb300._build.build()" % LIB)
        L = ctypes.CDLL(LIB)
        vp, i64, f64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        sig = {
            "airg_options_default": [ctypes.POINTER(airg_options)],
            "airg_problem_advection2d": [i64, i64, f64, f64, f64, vp, vp, vp, vp,
                                         ctypes.POINTER(i64), ctypes.POINTER(i64), vp],
            "airg_assemble_rhs_advection2d": [i64, i64, f64, f64, f64, ci, vp, i64, vp, vp, vp, vp],
            "airg_setup": [ctypes.POINTER(airg_csr), ctypes.POINTER(airg_options), vp,
                           ctypes.POINTER(vp)],
            "airg_solve": [vp, ci, vp, vp, ci, f64, f64, ci, ctypes.POINTER(airg_solve_info), vp],
            "airg_solve_adjoint": [vp, ci, vp, vp, ci, f64, f64, ci,
                                   ctypes.POINTER(airg_solve_info), vp],
            "airg_setup_info": [vp, ctypes.POINTER(airg_hierarchy_info)],
            "airg_batch_setup_info": [vp, ci, ctypes.POINTER(airg_hierarchy_info)],
            "airg_export_matrix": [vp, ci, ci, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                   ctypes.POINTER(i64), vp, vp, vp],
            "airg_export_vector": [vp, ci, ci, ctypes.POINTER(i64), vp],
            "airg_dot_exact": [i64, vp, vp, ctypes.POINTER(f64), vp],
            "airg_rng_uniform": [ctypes.c_uint64, i64, i64, i64, vp, vp],
            "airg_host_gmres_coeffs": [ci, vp, f64, vp],
            "airg_host_eigvals": [ci, vp, vp, vp],
            "airg_profile": [vp, ci],
            "airg_profile_group": [vp, ci, ci],
            "airg_batch_profile": [vp, ci],
            "airg_batch_profile_read": [vp, ctypes.POINTER(f64), ctypes.POINTER(i64), ctypes.POINTER(i64)],
            "airg_dot_exact_noalloc": [i64, vp, vp, vp, vp],
            "airg_rhs_adjoint_advection2d": [i64, i64, f64, f64, f64, ci, vp, i64, vp, vp, vp, vp],
            "airg_check_wait_timeout": [i64, vp],
            "airg_setup_batch": [ci, ctypes.POINTER(airg_csr), ctypes.POINTER(airg_options), vp,
                                 ctypes.POINTER(vp)],
            "airg_solve_batch": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ci, f64, f64, ci,
                                 ctypes.POINTER(airg_solve_info), vp],
            "airg_profile_read": [vp, ci, ctypes.POINTER(f64), ctypes.POINTER(i64),
                                  ctypes.POINTER(i64)],
            "airg_profile_read_level": [vp, ci, ci, ctypes.POINTER(f64), ctypes.POINTER(i64),
                                        ctypes.POINTER(i64), ctypes.POINTER(i64)],
            "airg_operator_layout_info": [vp, ci, ci, ctypes.POINTER(airg_operator_layout)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.airg_free.argtypes = [vp]
        L.airg_free.restype = None
        L.airg_batch_free.argtypes = [vp]
        L.airg_batch_free.restype = None
        L.airg_last_error.argtypes = []
        L.airg_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status, allow=()):
    if status != AIRG_OK and status not in allow:
        raise AirgError(status, airg_last_error())
    return status


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def airg_last_error():
    return lib().airg_last_error().decode()


def airg_options_default(**overrides):
    o = airg_options()
    _check(lib().airg_options_default(ctypes.byref(o)))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def airg_problem_advection2d(nx, ny, vx, vy, h=None, stream=None):
    """Device CSR (rowptr int64, col int32, val f64) and inflow node list.
    h = None: the library's default spacing of the unit square (passed as 0)."""
    import torch
    h = 0.0 if h is None else h
    n = nx * ny
    dev = torch.device("cuda")
    rowptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(3 * n, dtype=torch.int32, device=dev)
    val = torch.empty(3 * n, dtype=torch.float64, device=dev)
    inflow = torch.empty(nx + ny, dtype=torch.int64, device=dev)
    nnz, nin = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().airg_problem_advection2d(nx, ny, float(vx), float(vy), float(h), _ptr(rowptr),
                                          _ptr(col), _ptr(val), _ptr(inflow), ctypes.byref(nnz),
                                          ctypes.byref(nin), _stream(stream)))
    return {"rowptr": rowptr, "col": col[: nnz.value], "val": val[: nnz.value],
            "inflow": inflow[: nin.value], "n": n, "nx": nx, "ny": ny, "vx": vx, "vy": vy, "h": h}


def airg_assemble_rhs_advection2d(prob, g, s=None, stream=None):
    import torch
    nrhs = g.shape[0] if g.dim() == 2 else 1
    b = torch.empty(nrhs * prob["n"], dtype=torch.float64, device="cuda")
    g = g.contiguous()
    sp = _ptr(s.contiguous()) if s is not None else ctypes.c_void_p(0)
    _check(lib().airg_assemble_rhs_advection2d(prob["nx"], prob["ny"], float(prob["vx"]),
                                               float(prob["vy"]), float(prob["h"]), nrhs,
                                               _ptr(prob["inflow"]), prob["inflow"].numel(),
                                               _ptr(g), sp, _ptr(b), _stream(stream)))
    return b.view(nrhs, prob["n"]) if nrhs > 1 else b


def airg_rhs_adjoint_advection2d(prob, lam, want_s=True, stream=None):
    """(grad_g, grad_s) = (B^T lam, h lam off the inflow nodes) for one or
    more adjoint vectors lam (device, float64)."""
    import torch
    nrhs = lam.shape[0] if lam.dim() == 2 else 1
    nin = prob["inflow"].numel()
    gg = torch.empty(nrhs * nin, dtype=torch.float64, device="cuda")
    gs = torch.empty(nrhs * prob["n"], dtype=torch.float64, device="cuda") if want_s else None
    lam = lam.contiguous()
    _check(lib().airg_rhs_adjoint_advection2d(
        prob["nx"], prob["ny"], float(prob["vx"]), float(prob["vy"]), float(prob["h"]), nrhs,
        _ptr(prob["inflow"]), nin, _ptr(lam), _ptr(gg), _ptr(gs) if gs is not None else None,
        _stream(stream)))
    if nrhs > 1:
        return gg.view(nrhs, nin), (gs.view(nrhs, prob["n"]) if gs is not None else None)
    return gg, gs


class Handle:
    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        if getattr(self, "ptr", None):
            airg_free(self)


def airg_setup(rowptr, col, val, opts=None, stream=None):
    """rowptr/col/val: torch tensors (CUDA or CPU) of a square CSR matrix."""
    on_dev = int(rowptr.is_cuda)
    A = airg_csr(rowptr.numel() - 1, rowptr.numel() - 1, col.numel(), rowptr.data_ptr(),
                 col.data_ptr(), val.data_ptr(), on_dev)
    out = ctypes.c_void_p()
    o = opts if opts is not None else airg_options_default()
    _check(lib().airg_setup(ctypes.byref(A), ctypes.byref(o), _stream(stream), ctypes.byref(out)))
    return Handle(out)


def _solve(fn, handle, b, x, rtol, atol, maxit, stream, allow_nc):
    import torch
    on_dev = int(b.is_cuda)
    nrhs = b.shape[0] if b.dim() == 2 else 1
    if x is None:
        x = torch.zeros_like(b)
    info = airg_solve_info()
    st = fn(handle.ptr, nrhs, _ptr(b), _ptr(x), on_dev, float(rtol), float(atol), int(maxit),
            ctypes.byref(info), _stream(stream))
    _check(st, allow=(AIRG_ERR_NOT_CONVERGED,) if allow_nc else ())
    return x, info


class BatchHandle:
    def __init__(self, ptr, sizes):
        self.ptr = ptr
        self.sizes = sizes

    def __del__(self):
        if getattr(self, "ptr", None):
            airg_batch_free(self)


def airg_setup_batch(csrs, opts=None, stream=None):
    """csrs: list of (rowptr, col, val) tensors, one square matrix per problem."""
    n = len(csrs)
    arr = (airg_csr * n)()
    for i, (rp, ci_, v) in enumerate(csrs):
        arr[i] = airg_csr(rp.numel() - 1, rp.numel() - 1, ci_.numel(), rp.data_ptr(), ci_.data_ptr(),
                          v.data_ptr(), int(rp.is_cuda))
    out = ctypes.c_void_p()
    o = opts if opts is not None else airg_options_default()
    _check(lib().airg_setup_batch(n, arr, ctypes.byref(o), _stream(stream), ctypes.byref(out)))
    return BatchHandle(out, [rp.numel() - 1 for rp, _, _ in csrs])


def airg_solve_batch(batch, bs, xs=None, rtol=1e-10, atol=1e-50, maxit=200, stream=None,
                     allow_nc=False):
    """Solves every problem of the batch; bs, xs: lists of tensors (same device)."""
    import torch
    n = len(bs)
    if xs is None:
        xs = [torch.zeros_like(b) for b in bs]
    pb = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    px = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    infos = (airg_solve_info * n)()
    st = lib().airg_solve_batch(batch.ptr, pb, px, int(bs[0].is_cuda), float(rtol), float(atol),
                                int(maxit), infos, _stream(stream))
    _check(st, allow=(AIRG_ERR_NOT_CONVERGED,) if allow_nc else ())
    return xs, list(infos)


def airg_batch_profile(batch, enable):
    _check(lib().airg_batch_profile(batch.ptr, int(enable)))


def airg_batch_profile_read(batch):
    """(ms, launches, algorithmic bytes) of the timed iteration launches."""
    ms, nl, nb = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().airg_batch_profile_read(batch.ptr, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(nb)))
    return ms.value, nl.value, nb.value


def airg_batch_free(batch):
    if batch.ptr:
        lib().airg_batch_free(batch.ptr)
        batch.ptr = None


def airg_solve(handle, b, x=None, rtol=1e-10, atol=1e-50, maxit=200, stream=None, allow_nc=False):
    """x (in/out, same device as b) and airg_solve_info."""
    return _solve(lib().airg_solve, handle, b, x, rtol, atol, maxit, stream, allow_nc)


def airg_solve_adjoint(handle, rhs, lam=None, rtol=1e-10, atol=1e-50, maxit=200, stream=None,
                       allow_nc=False):
    return _solve(lib().airg_solve_adjoint, handle, rhs, lam, rtol, atol, maxit, stream, allow_nc)


def airg_setup_info(handle):
    info = airg_hierarchy_info()
    _check(lib().airg_setup_info(handle.ptr, ctypes.byref(info)))
    return _info_dict(info)


def airg_batch_setup_info(batch, i):
    """airg_setup_info of problem i of a batch."""
    info = airg_hierarchy_info()
    _check(lib().airg_batch_setup_info(batch.ptr, int(i), ctypes.byref(info)))
    return _info_dict(info)


def _info_dict(info):
    L = info.levels
    return {"levels": L, "truncated": bool(info.truncated), "coarse_roots": info.coarse_roots,
            "coarse_krylov": info.coarse_krylov,
            "cycle_complexity": info.cycle_complexity,
            "storage_complexity": info.storage_complexity, "setup_ms": info.setup_ms,
            "n": list(info.n[:L]), "n_f": list(info.n_f[:L]), "nnz_a": list(info.nnz_a[:L]),
            "bytes_per_vcycle": info.bytes_per_vcycle,
            "setup_breakdown_ms": {k: info.setup_phase_ms[i] for i, k in enumerate(SETUP_PHASES)},
            "exact_dots": info.exact_dots}


def airg_export_matrix(handle, level, what):
    """(n_rows, n_cols, rowptr, col, val) as numpy arrays, level numbering."""
    nr, nc, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    L = lib()
    _check(L.airg_export_matrix(handle.ptr, level, what, ctypes.byref(nr), ctypes.byref(nc),
                                ctypes.byref(nnz), None, None, None))
    rp = np.empty(nr.value + 1, np.int64)
    ci = np.empty(max(nnz.value, 1), np.int32)
    v = np.empty(max(nnz.value, 1), np.float64)
    _check(L.airg_export_matrix(handle.ptr, level, what, ctypes.byref(nr), ctypes.byref(nc),
                                ctypes.byref(nnz), rp.ctypes.data, ci.ctypes.data, v.ctypes.data))
    return nr.value, nc.value, rp, ci[: nnz.value], v[: nnz.value]


_VEC_DTYPES = {0: np.int8, 1: np.int32, 2: np.float64, 3: np.float64, 4: np.float64, 5: np.float64}


def airg_export_vector(handle, level, what):
    cnt = ctypes.c_int64()
    L = lib()
    _check(L.airg_export_vector(handle.ptr, level, what, ctypes.byref(cnt), None))
    out = np.empty(max(cnt.value, 1), _VEC_DTYPES[what])
    _check(L.airg_export_vector(handle.ptr, level, what, ctypes.byref(cnt), out.ctypes.data))
    return out[: cnt.value]


def airg_check_wait_timeout(spin_limit=20000, stream=None):
    """Status of the bounded-wait self check (AIRG_ERR_TIMEOUT = 6 is the
    designed outcome)."""
    return lib().airg_check_wait_timeout(int(spin_limit), _stream(stream))


def airg_free(handle):
    if handle.ptr:
        lib().airg_free(handle.ptr)
        handle.ptr = None


def airg_profile(handle, enable):
    _check(lib().airg_profile(handle.ptr, int(enable)))


def airg_profile_group(handle, kind, level):
    """Time only the launches of one (kernel kind, level) group; kind is a
    name of PROFILE_KINDS or its index."""
    k = PROFILE_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    _check(lib().airg_profile_group(handle.ptr, k, int(level)))


def airg_profile_read(handle):
    """{kind: (ms, launches, algorithmic bytes)} for every kernel kind."""
    out = {}
    for k, name in enumerate(PROFILE_KINDS):
        ms, nl, nb = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().airg_profile_read(handle.ptr, k, ctypes.byref(ms), ctypes.byref(nl),
                                       ctypes.byref(nb)))
        out[name] = (ms.value, nl.value, nb.value)
    return out


def airg_profile_read_level(handle, levels):
    """{(kind, level): (ms, launches, algorithmic bytes, flops)} for levels <
    `levels`, entries with launches only."""
    out = {}
    for k, name in enumerate(PROFILE_KINDS):
        for lev in range(levels):
            ms, nl, nb, nf = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
            _check(lib().airg_profile_read_level(handle.ptr, k, lev, ctypes.byref(ms), ctypes.byref(nl),
                                                 ctypes.byref(nb), ctypes.byref(nf)))
            if nl.value:
                out[(name, lev)] = (ms.value, nl.value, nb.value, nf.value)
    return out


def airg_operator_layout_info(handle, level, op):
    """Layout and tuned row-kernel variant of operator `op` (an index or a
    name of OPERATORS) of `level`, as a dict; n_rows 0 for an operator the
    hierarchy does not keep."""
    if isinstance(op, str):
        op = OPERATORS.index(op)
    out = airg_operator_layout()
    _check(lib().airg_operator_layout_info(handle.ptr, int(level), int(op), ctypes.byref(out)))
    return {name: getattr(out, name) for name, _ in airg_operator_layout._fields_}


def airg_row_kernel_choices(handle):
    """Every operator that the solve keeps, level by level:
    [(level, name, layout dict)]."""
    L = airg_setup_info(handle)["levels"] - 1
    rows = [(0, "top", airg_operator_layout_info(handle, 0, "top"))]
    for lev in range(L):
        for name in OPERATORS[1:-1]:
            d = airg_operator_layout_info(handle, lev, name)
            if d["n_rows"]:
                rows.append((lev, name, d))
    rows.append((L, "coarse", airg_operator_layout_info(handle, L, "coarse")))
    return rows


def _dev_f64(t, name):
    """Rejects anything but a contiguous float64 CUDA tensor (the C entry
    points read raw device addresses and cannot check them)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda \
            or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)


def _dot_operands(x, y):
    _dev_f64(x, "x")
    _dev_f64(y, "y")
    if x.numel() != y.numel():
        raise ValueError("x and y differ in length (%d, %d)" % (x.numel(), y.numel()))
    return x.numel()


def airg_dot_exact(x, y, stream=None):
    n = _dot_operands(x, y)
    out = ctypes.c_double()
    _check(lib().airg_dot_exact(n, _ptr(x), _ptr(y), ctypes.byref(out), _stream(stream)))
    return out.value


def airg_dot_exact_noalloc(x, y, out, stream=None):
    """Correctly rounded <x, y> into the device tensor `out` (one double),
    without any device allocation; asynchronous on the stream."""
    n = _dot_operands(x, y)
    _dev_f64(out, "out")
    if out.numel() < 1:
        raise ValueError("out must hold one element")
    _check(lib().airg_dot_exact_noalloc(n, _ptr(x), _ptr(y), _ptr(out), _stream(stream)))


def airg_rng_uniform(seed, level, purpose, n, stream=None):
    import torch
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    _check(lib().airg_rng_uniform(seed, level, purpose, n, _ptr(out), _stream(stream)))
    return out


def airg_host_gmres_coeffs(H, beta):
    H = np.ascontiguousarray(H, dtype=np.float64)
    k = H.shape[1]
    alpha = np.empty(k)
    _check(lib().airg_host_gmres_coeffs(k, H.ctypes.data, float(beta), alpha.ctypes.data))
    return alpha


def airg_host_eigvals(H):
    H = np.ascontiguousarray(H, dtype=np.float64)
    n = H.shape[0]
    wr, wi = np.empty(n), np.empty(n)
    _check(lib().airg_host_eigvals(n, H.ctypes.data, wr.ctypes.data, wi.ctypes.data))
    return wr + 1j * wi


# ---------------------------------------------------------------- autograd --
def _make_autograd():
    import torch

    class AdvectionSolveFn(torch.autograd.Function):
        """u = A^-1 (B g + h s) with gradients by one adjoint AIRG solve on
        A^T: dL/dg = B^T lambda, dL/ds = h lambda (inflow rows excluded),
        lambda = A^-T dL/du."""

        @staticmethod
        def forward(ctx, g, s, solver, rtol):
            u = solver.solve_plain(g, s, rtol)
            ctx.solver, ctx.rtol, ctx.s_dtype = solver, rtol, s.dtype
            return u

        @staticmethod
        def backward(ctx, gu):
            lam, _ = airg_solve_adjoint(ctx.solver.handle, gu.contiguous().double(), rtol=ctx.rtol)
            gg, gs = airg_rhs_adjoint_advection2d(ctx.solver.prob, lam)
            return gg, gs.to(ctx.s_dtype), None, None

    return AdvectionSolveFn


class AdvectionSolver:
    """The upwind advection problem of Eq. 1-2 on an nx-by-ny grid with an
    AIRG hierarchy; solve(g, s) is differentiable in the inflow values g
    (float64) and the source s (float32 or float64) through the adjoint."""

    def __init__(self, nx, ny, vx, vy, h=None, opts=None):
        self.prob = airg_problem_advection2d(nx, ny, vx, vy, h)
        p = self.prob
        self.handle = airg_setup(p["rowptr"], p["col"], p["val"], opts)
        self._fn = None

    def solve_plain(self, g, s=None, rtol=1e-10):
        sd = s.double() if s is not None else None
        b = airg_assemble_rhs_advection2d(self.prob, g.double(), sd)
        u, info = airg_solve(self.handle, b, rtol=rtol)
        return u

    def solve(self, g, s, rtol=1e-10):
        if self._fn is None:
            self._fn = _make_autograd()
        return self._fn.apply(g, s, self, rtol)
