"""AIRG oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct CPU FP64 restatement of the AIRG reduction
multigrid (Dargaville et al., "Solving advection equations with reduction
multigrids on GPUs", arXiv 2508.17517) for the 2D upwind advection operator.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
in ``paper_2508_17517_gb300``: neither imports the other.

``build()`` compiles ``airg_oracle.c`` with gcc (-O2 -ffp-contract=off) into
``oracle/_build/liboracle.so``; ``lib()`` loads it with ctypes.
"""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "airg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle's C kernels (plain gcc, no vectorising flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        so = build()
        L = ctypes.CDLL(so)
        i64, f64, vp, u64 = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_uint64
        L.orc_rng_key.restype = u64
        L.orc_rng_key.argtypes = [u64, i64, i64]
        L.orc_rng_uniform.argtypes = [u64, i64, vp]
        L.orc_rng_u32.argtypes = [u64, i64, vp]
        L.orc_dot_exact.restype = f64
        L.orc_dot_exact.argtypes = [i64, vp, vp]
        L.orc_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
        L.orc_strength.argtypes = [i64, vp, vp, vp, f64, vp]
        L.orc_ddc_ratio.argtypes = [i64, vp, vp, vp, vp, vp]
        L.orc_fixed_sparsity_power.argtypes = [i64, vp, vp, vp, vp, vp]
        L.orc_spgemm.restype = ctypes.c_int
        L.orc_spgemm.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp,
                                 ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.orc_free.argtypes = [vp]
        L.orc_drop_lump.restype = ctypes.c_int
        L.orc_drop_lump.argtypes = [i64, vp, vp, vp, f64, ctypes.c_int, vp, vp]
        L.orc_drop_rows.argtypes = [i64, vp, vp, f64, vp]
        L.orc_one_point.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
        L.orc_sweep.restype = ctypes.c_int
        L.orc_sweep.argtypes = [i64, vp, vp, vp, vp, vp, vp]
        _lib = L
    return _lib
