"""The allocation-free grouped entry point (iaat_gemm_grouped_noalloc).

Some callers cannot allocate device memory once they are running -- a
serving process that reserved all GPU memory at start-up, for instance, and
treats any later cudaMalloc as a failure because cudaMalloc and cudaFree
synchronise the device and can fail under memory pressure.  For them the
library has one entry point that plans into static host arrays and runs from
a fixed device scratch array.  These tests call it through the C ABI and
check that two calls in a row give the same C as the regular planned entry
point (iaat_plan_create + iaat_gemm_grouped), within the 1e-5 / 1e-13
normwise bound the other tests use.  This file is collected last.
"""
import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

from .gpu_util import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_09822_gb300 import build
    build.build()
    iaat.lib()
    return torch


@pytest.mark.parametrize("dtype,tol", [(np.float32, 1e-5), (np.float64, 1e-13)])
def test_noalloc_matches_planned_entry_point_twice(cuda, dtype, tol):
    torch = cuda
    b = W.random_small(3000, seed=77, dtype=dtype, max_dim=80, pad_max=3, misalign_max=1)
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    tA, tB, tC, descs = to_device(b)
    C0 = tC.clone()
    ddt = iaat.IAAT_F32 if dtype == np.float32 else iaat.IAAT_F64
    s = torch.cuda.current_stream()
    plan = iaat.iaat_plan_create(descs, ddt)
    iaat.iaat_gemm_grouped(plan, s)
    iaat.iaat_plan_check(plan, s)
    ref = tC.cpu().numpy().astype(np.float64)
    plan.destroy()
    for call in range(2):
        tC.copy_(C0)
        iaat.iaat_gemm_grouped_noalloc(descs, ddt, s)
        iaat.iaat_plan_check(None, s)
        got = tC.cpu().numpy().astype(np.float64)
        fin = np.isfinite(ref)
        assert np.array_equal(np.isnan(got), np.isnan(ref)), call
        err = np.linalg.norm(got[fin] - ref[fin]) / np.linalg.norm(ref[fin])
        assert err <= tol, (call, err)


def test_noalloc_rejects_too_many_tasks(cuda):
    d = np.zeros(8193, iaat.DESC_DTYPE)
    for k, v in dict(M=1, N=1, K=1, lda=1, ldb=1, ldc=1, alpha=1.0, beta=0.0, A=0x1000, B=0x2000,
                     C=0x3000).items():
        d[k] = v
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_gemm_grouped_noalloc(d, iaat.IAAT_F32)
    assert e.value.status == 1 and "8192" in e.value.message
