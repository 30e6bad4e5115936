"""ctypes binding of libiaat.so (include/iaat.h): argument marshalling only.

Every GEMM runs in the library's CUDA kernels; nothing here computes.  If the
library is missing, the first call raises -- there is no fallback.
Pointers are passed as integers (device addresses, e.g. from
``torch.Tensor.data_ptr()``); streams as integer handles
(``torch.cuda.Stream.cuda_stream``) or None for the legacy default stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiaat.so")

IAAT_OP_N, IAAT_OP_T = 0, 1
IAAT_F32, IAAT_F64, IAAT_C32, IAAT_C64 = 0, 1, 2, 3
IAAT_PREC_DEFAULT, IAAT_PREC_3XBF16, IAAT_PREC_TF32, IAAT_PREC_FP16, IAAT_PREC_6XBF16 = 0, 1, 2, 3, 4
STATUS = {0: "IAAT_OK", 1: "IAAT_ERR_INVALID_VALUE", 2: "IAAT_ERR_NOT_SMALL", 3: "IAAT_ERR_MISALIGNED",
          4: "IAAT_ERR_UNSUPPORTED", 5: "IAAT_ERR_CUDA", 6: "IAAT_ERR_DEVICE_TIMEOUT", 7: "IAAT_ERR_OOM"}

#: numpy mirror of iaat_gemm_desc_t (72 bytes)
DESC_DTYPE = np.dtype([("M", "<i4"), ("N", "<i4"), ("K", "<i4"), ("lda", "<i4"), ("ldb", "<i4"),
                       ("ldc", "<i4"), ("transA", "<i4"), ("transB", "<i4"), ("alpha", "<f8"),
                       ("beta", "<f8"), ("A", "<u8"), ("B", "<u8"), ("C", "<u8")])
assert DESC_DTYPE.itemsize == 72

#: numpy mirror of iaat_cgemm_desc_t (88 bytes)
CDESC_DTYPE = np.dtype([("M", "<i4"), ("N", "<i4"), ("K", "<i4"), ("lda", "<i4"), ("ldb", "<i4"),
                        ("ldc", "<i4"), ("transA", "<i4"), ("transB", "<i4"), ("alpha_re", "<f8"),
                        ("alpha_im", "<f8"), ("beta_re", "<f8"), ("beta_im", "<f8"), ("A", "<u8"),
                        ("B", "<u8"), ("C", "<u8")])
assert CDESC_DTYPE.itemsize == 88


class IaatError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class PlanOptions(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("max_group_tasks", ctypes.c_int32),
                ("force_variant", ctypes.c_int32), ("inject_fault", ctypes.c_int32),
                ("route_k_below", ctypes.c_int32), ("kernel", ctypes.c_int32), ("route_mnk_below", ctypes.c_int32),
                ("route_kernel", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int64), ("active", ctypes.c_int64), ("tasks", ctypes.c_int64),
                ("groups", ctypes.c_int64), ("blocks", ctypes.c_int64), ("flops", ctypes.c_int64),
                ("algorithmic_bytes", ctypes.c_int64), ("plan_bytes", ctypes.c_int64),
                ("grid", ctypes.c_int32), ("kernels", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("kernel_family", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None


def lib():
    """The loaded libiaat.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2208_09822_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        I, P, D, F, S = ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_float, ctypes.c_int
        L.iaat_sgemm.restype = S
        L.iaat_sgemm.argtypes = [I, I, I, I, I, F, P, I, P, I, F, P, I, P]
        L.iaat_dgemm.restype = S
        L.iaat_dgemm.argtypes = [I, I, I, I, I, D, P, I, P, I, D, P, I, P]
        L.iaat_cgemm.restype = S
        L.iaat_cgemm.argtypes = [I, I, I, I, I, ctypes.POINTER(F), P, I, P, I, ctypes.POINTER(F), P, I, P]
        L.iaat_zgemm.restype = S
        L.iaat_zgemm.argtypes = [I, I, I, I, I, ctypes.POINTER(D), P, I, P, I, ctypes.POINTER(D), P, I, P]
        L.iaat_plan_create.restype = S
        L.iaat_plan_create.argtypes = [P, ctypes.c_int64, I, I, ctypes.POINTER(PlanOptions),
                                       ctypes.POINTER(ctypes.c_void_p)]
        L.iaat_plan_create_complex.restype = S
        L.iaat_plan_create_complex.argtypes = [P, ctypes.c_int64, I, ctypes.POINTER(PlanOptions),
                                               ctypes.POINTER(ctypes.c_void_p)]
        L.iaat_pack_create.restype = S
        L.iaat_pack_create.argtypes = [P, ctypes.c_int64, I, P, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_void_p)]
        L.iaat_pack_run.restype = S
        L.iaat_pack_run.argtypes = [P, P]
        L.iaat_pack_destroy.restype = S
        L.iaat_pack_destroy.argtypes = [P]
        L.iaat_gemm_grouped_noalloc.restype = S
        L.iaat_gemm_grouped_noalloc.argtypes = [P, ctypes.c_int64, I, P]
        L.iaat_gemm_grouped.restype = S
        L.iaat_gemm_grouped.argtypes = [P, P]
        L.iaat_plan_check.restype = S
        L.iaat_plan_check.argtypes = [P, P]
        L.iaat_plan_info.restype = S
        L.iaat_plan_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
        L.iaat_plan_destroy.restype = S
        L.iaat_plan_destroy.argtypes = [P]
        L.iaat_autotune.restype = S
        L.iaat_autotune.argtypes = [I, I, ctypes.c_char_p]
        L.iaat_fma_peak.restype = S
        L.iaat_fma_peak.argtypes = [I, ctypes.POINTER(ctypes.c_double)]
        L.iaat_tile.restype = ctypes.c_int64
        L.iaat_tile.argtypes = [I, I, I, I, I, I, P, ctypes.c_int64]
        L.iaat_tile_exact.restype = ctypes.c_int64
        L.iaat_tile_exact.argtypes = [I, I, P, P, I, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        L.iaat_version.restype = ctypes.c_char_p
        L.iaat_version.argtypes = []
        L.iaat_last_error.restype = ctypes.c_char_p
        L.iaat_last_error.argtypes = []
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise IaatError(status, iaat_last_error())


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def iaat_version():
    return lib().iaat_version().decode()


def iaat_last_error():
    return lib().iaat_last_error().decode()


def iaat_sgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    _check(lib().iaat_sgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, _stream(stream)))


def iaat_dgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    _check(lib().iaat_dgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, _stream(stream)))


def iaat_cgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    """Single complex-float GEMM; alpha and beta are Python complex numbers."""
    al = (ctypes.c_float * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ctypes.c_float * 2)(complex(beta).real, complex(beta).imag)
    _check(lib().iaat_cgemm(transA, transB, M, N, K, al, A, lda, B, ldb, be, C, ldc, _stream(stream)))


def iaat_zgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    """Single complex-double GEMM; alpha and beta are Python complex numbers."""
    al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
    _check(lib().iaat_zgemm(transA, transB, M, N, K, al, A, lda, B, ldb, be, C, ldc, _stream(stream)))


class Plan:
    """Owner of an iaat_plan_t; destroyed with the object."""

    def __init__(self, handle, keepalive=None):
        self.handle = handle
        self._keep = keepalive

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self):
        if self.handle:
            lib().iaat_plan_destroy(self.handle)
            self.handle = None


def iaat_plan_create(descs, dtype, precision=IAAT_PREC_DEFAULT, *, max_group_tasks=0, force_variant=0,
                     inject_fault=0, route_k_below=0, kernel=0, route_mnk_below=0, route_kernel=0):
    """descs: numpy array of DESC_DTYPE (device pointers inside).  kernel
    (iaat_plan_options_t.kernel): 0 = default, 1 = stage-program kernels,
    2 = stream kernels, 3 = warp-tile tensor-core kernel, 4 = warp-direct
    CUDA-core kernel; route_kernel: the family of a routed plan's CUDA-core
    part."""
    descs = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
    opts = PlanOptions(0, max_group_tasks, force_variant, inject_fault, route_k_below, kernel, route_mnk_below,
                       route_kernel)
    h = ctypes.c_void_p()
    _check(lib().iaat_plan_create(descs.ctypes.data if len(descs) else None, len(descs), dtype, precision,
                                  ctypes.byref(opts), ctypes.byref(h)))
    return Plan(h.value)


def iaat_plan_create_complex(descs, dtype, *, max_group_tasks=0, force_variant=0, inject_fault=0):
    """descs: numpy array of CDESC_DTYPE (device pointers inside); dtype
    IAAT_C32 or IAAT_C64."""
    descs = np.ascontiguousarray(descs, dtype=CDESC_DTYPE)
    opts = PlanOptions(0, max_group_tasks, force_variant, inject_fault)
    h = ctypes.c_void_p()
    _check(lib().iaat_plan_create_complex(descs.ctypes.data if len(descs) else None, len(descs), dtype,
                                          ctypes.byref(opts), ctypes.byref(h)))
    return Plan(h.value)


class Pack:
    """Owner of an iaat_pack_t (the ablation's pack step); destroyed with the
    object.  ``packed`` holds the descriptors of the packed instances and
    ``bytes_moved`` the pack kernel's algorithmic bytes per run."""

    def __init__(self, handle, packed, bytes_moved):
        self.handle = handle
        self.packed = packed
        self.bytes_moved = bytes_moved

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self):
        if self.handle:
            lib().iaat_pack_destroy(self.handle)
            self.handle = None


def iaat_pack_create(descs, dtype):
    descs = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
    packed = np.zeros(len(descs), DESC_DTYPE)
    moved = ctypes.c_int64()
    h = ctypes.c_void_p()
    _check(lib().iaat_pack_create(descs.ctypes.data if len(descs) else None, len(descs), dtype,
                                  packed.ctypes.data if len(descs) else None, ctypes.byref(moved),
                                  ctypes.byref(h)))
    return Pack(h.value, packed, moved.value)


def iaat_pack_run(pack, stream=None):
    _check(lib().iaat_pack_run(pack.handle, _stream(stream)))


def iaat_gemm_grouped_noalloc(descs, dtype, stream=None):
    """Allocation-free grouped GEMM (see include/iaat.h): descs is a
    DESC_DTYPE array with device pointers inside."""
    descs = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
    _check(lib().iaat_gemm_grouped_noalloc(descs.ctypes.data if len(descs) else None, len(descs), dtype,
                                           _stream(stream)))


def iaat_gemm_grouped(plan, stream=None):
    _check(lib().iaat_gemm_grouped(plan.handle, _stream(stream)))


def iaat_plan_check(plan, stream=None):
    _check(lib().iaat_plan_check(plan.handle if plan is not None else None, _stream(stream)))


def iaat_plan_info(plan):
    info = PlanInfo()
    _check(lib().iaat_plan_info(plan.handle, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in PlanInfo._fields_}


def iaat_plan_destroy(plan):
    plan.destroy()


def iaat_autotune(dtype, precision=IAAT_PREC_DEFAULT, cache_path=None):
    _check(lib().iaat_autotune(dtype, precision, cache_path.encode() if cache_path else None))


def iaat_fma_peak(dtype):
    """FMA-pipe throughput of the current GPU in GFLOP/s."""
    v = ctypes.c_double()
    _check(lib().iaat_fma_peak(dtype, ctypes.byref(v)))
    return v.value


def iaat_tile(dtype, transA, transB, M, N, K):
    n = lib().iaat_tile(dtype, transA, transB, M, N, K, None, 0)
    if n < 0:
        raise ValueError("iaat_tile rejected its arguments")
    buf = np.zeros(max(1, 4 * n), np.int32)
    lib().iaat_tile(dtype, transA, transB, M, N, K, buf.ctypes.data, n)
    return [tuple(int(x) for x in buf[4 * i:4 * i + 4]) for i in range(n)]


def iaat_tile_exact(M, N, heights, max_widths):
    h = np.ascontiguousarray(heights, np.int32)
    w = np.ascontiguousarray(max_widths, np.int32)
    s = ctypes.c_int64()
    n = lib().iaat_tile_exact(M, N, h.ctypes.data, w.ctypes.data, len(h), None, 0, ctypes.byref(s))
    if n < 0:
        raise ValueError("no exact cover")
    buf = np.zeros(max(1, 4 * n), np.int32)
    lib().iaat_tile_exact(M, N, h.ctypes.data, w.ctypes.data, len(h), buf.ctypes.data, n, ctypes.byref(s))
    return [tuple(int(x) for x in buf[4 * i:4 * i + 4]) for i in range(n)], int(s.value)


def descs_for_pools(batch, baseA, baseB, baseC):
    """iaat_gemm_desc_t array for a workloads.Batch whose pools sit at device
    addresses baseA/baseB/baseC."""
    d = np.zeros(batch.count, dtype=DESC_DTYPE)
    for f in ("M", "N", "K", "lda", "ldb", "ldc"):
        d[f] = getattr(batch, f)
    d["transA"] = batch.transA
    d["transB"] = batch.transB
    d["alpha"] = batch.alpha
    d["beta"] = batch.beta
    esz = batch.esize
    d["A"] = np.uint64(baseA) + batch.offA.astype(np.uint64) * np.uint64(esz)
    d["B"] = np.uint64(baseB) + batch.offB.astype(np.uint64) * np.uint64(esz)
    d["C"] = np.uint64(baseC) + batch.offC.astype(np.uint64) * np.uint64(esz)
    return d


def cdescs_for_pools(batch, baseA, baseB, baseC):
    """iaat_cgemm_desc_t array for a complex workloads.Batch whose pools sit
    at device addresses baseA/baseB/baseC."""
    d = np.zeros(batch.count, dtype=CDESC_DTYPE)
    for f in ("M", "N", "K", "lda", "ldb", "ldc"):
        d[f] = getattr(batch, f)
    d["transA"] = batch.transA
    d["transB"] = batch.transB
    al = np.asarray(batch.alpha, np.complex128)
    be = np.asarray(batch.beta, np.complex128)
    d["alpha_re"], d["alpha_im"] = al.real, al.imag
    d["beta_re"], d["beta_im"] = be.real, be.imag
    esz = batch.esize
    d["A"] = np.uint64(baseA) + batch.offA.astype(np.uint64) * np.uint64(esz)
    d["B"] = np.uint64(baseB) + batch.offB.astype(np.uint64) * np.uint64(esz)
    d["C"] = np.uint64(baseC) + batch.offC.astype(np.uint64) * np.uint64(esz)
    return d
