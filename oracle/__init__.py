"""FP64 CPU oracle for small-GEMM batches -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_2208_09822_gb300/`` never imports it, and it imports nothing from the
library: the two share only the seeded input generators, which hold none of
the GEMM arithmetic.

* ``gemm_oracle.c``   -- the GEMM definition (Sec. I; Table I note for the
  transposition names and column-major storage) as an FP64 triple loop, for
  real and for complex (CGEMM/ZGEMM, Table I rows 3-4) batches.
* ``tiler_oracle.py`` -- Algorithm 2 (Sec. V-A) and the memops count.
* ``split_oracle.py`` -- the steps of the tensor-core paths (operand
  rounding to BF16 terms, TF32 or FP16, and their product sets) in FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gemm_oracle.c")


def lib_path(mutant=0):
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_HERE, name)


def build(mutant=0, force=False):
    """Compile gemm_oracle.c into a shared library (gcc, OpenMP)."""
    out = lib_path(mutant)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           f"-DORACLE_MUTANT={int(mutant)}", _SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


_libs = {}


def _load(mutant=0):
    if mutant not in _libs:
        lib = ctypes.CDLL(build(mutant))
        p = ctypes.c_void_p
        lib.oracle_gemm_batch.restype = ctypes.c_int
        lib.oracle_gemm_batch.argtypes = [ctypes.c_int64, ctypes.c_int] + [p] * 18 + [ctypes.c_int]
        lib.oracle_cgemm_batch.restype = ctypes.c_int
        lib.oracle_cgemm_batch.argtypes = [ctypes.c_int64, ctypes.c_int] + [p] * 18 + [ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        _libs[mutant] = lib
    return _libs[mutant]


def max_threads():
    return _load().oracle_max_threads()


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def gemm_batch(batch, idx=None, nthreads=0, mutant=0):
    """Run the oracle on instances ``idx`` (all when None) of a
    ``workloads.Batch``.  Returns (out, off): the FP64 results, instance t's
    tight MxN column-major block at out[off[j]:...] for the j-th selected
    instance."""
    lib = _load(mutant)
    if idx is None:
        idx = np.arange(batch.count)
    idx = np.asarray(idx, dtype=np.int64)
    Ms = np.ascontiguousarray(batch.M[idx], dtype=np.int32)
    Ns = np.ascontiguousarray(batch.N[idx], dtype=np.int32)
    sizes = Ms.astype(np.int64) * Ns.astype(np.int64)
    off = np.zeros(len(idx), dtype=np.int64)
    if len(idx) > 1:
        off[1:] = np.cumsum(sizes)[:-1]
    out = np.zeros(int(sizes.sum()) if len(idx) else 0, dtype=np.float64)
    cols = [np.ascontiguousarray(a[idx]) for a in (
        batch.K, batch.lda, batch.ldb, batch.ldc)]
    cols = [c.astype(np.int32) for c in cols]
    ta = np.ascontiguousarray(batch.transA[idx], dtype=np.uint8)
    tb = np.ascontiguousarray(batch.transB[idx], dtype=np.uint8)
    al = np.ascontiguousarray(batch.alpha[idx], dtype=np.float64)
    be = np.ascontiguousarray(batch.beta[idx], dtype=np.float64)
    oA = np.ascontiguousarray(batch.offA[idx], dtype=np.int64)
    oB = np.ascontiguousarray(batch.offB[idx], dtype=np.int64)
    oC = np.ascontiguousarray(batch.offC[idx], dtype=np.int64)
    is_f64 = 1 if batch.A.dtype == np.float64 else 0
    rc = lib.oracle_gemm_batch(
        len(idx), is_f64, _ptr(Ms), _ptr(Ns), _ptr(cols[0]), _ptr(cols[1]),
        _ptr(cols[2]), _ptr(cols[3]), _ptr(ta), _ptr(tb), _ptr(al), _ptr(be),
        _ptr(batch.A), _ptr(oA), _ptr(batch.B), _ptr(oB), _ptr(batch.C),
        _ptr(oC), _ptr(out), _ptr(off), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the batch (negative size)")
    return out, off


def cgemm_batch(batch, idx=None, nthreads=0, mutant=0):
    """Complex counterpart of ``gemm_batch`` for a batch whose pools are
    complex64 (CGEMM) or complex128 (ZGEMM): returns (out, off) with ``out``
    complex128, instance j's tight MxN column-major block at out[off[j]:...]."""
    lib = _load(mutant)
    if idx is None:
        idx = np.arange(batch.count)
    idx = np.asarray(idx, dtype=np.int64)
    Ms = np.ascontiguousarray(batch.M[idx], dtype=np.int32)
    Ns = np.ascontiguousarray(batch.N[idx], dtype=np.int32)
    sizes = Ms.astype(np.int64) * Ns.astype(np.int64)
    off = np.zeros(len(idx), dtype=np.int64)
    if len(idx) > 1:
        off[1:] = np.cumsum(sizes)[:-1]
    out = np.zeros(int(sizes.sum()) if len(idx) else 0, dtype=np.complex128)
    cols = [np.ascontiguousarray(a[idx]).astype(np.int32) for a in (
        batch.K, batch.lda, batch.ldb, batch.ldc)]
    ta = np.ascontiguousarray(batch.transA[idx], dtype=np.uint8)
    tb = np.ascontiguousarray(batch.transB[idx], dtype=np.uint8)
    al = np.ascontiguousarray(batch.alpha[idx], dtype=np.complex128)
    be = np.ascontiguousarray(batch.beta[idx], dtype=np.complex128)
    oA = np.ascontiguousarray(batch.offA[idx], dtype=np.int64)
    oB = np.ascontiguousarray(batch.offB[idx], dtype=np.int64)
    oC = np.ascontiguousarray(batch.offC[idx], dtype=np.int64)
    if batch.A.dtype == np.complex128:
        is_c64 = 1
    elif batch.A.dtype == np.complex64:
        is_c64 = 0
    else:
        raise TypeError("cgemm_batch needs complex64 or complex128 pools")
    rc = lib.oracle_cgemm_batch(
        len(idx), is_c64, _ptr(Ms), _ptr(Ns), _ptr(cols[0]), _ptr(cols[1]),
        _ptr(cols[2]), _ptr(cols[3]), _ptr(ta), _ptr(tb), _ptr(al), _ptr(be),
        _ptr(batch.A), _ptr(oA), _ptr(batch.B), _ptr(oB), _ptr(batch.C),
        _ptr(oC), _ptr(out), _ptr(off), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the batch (negative size)")
    return out, off
