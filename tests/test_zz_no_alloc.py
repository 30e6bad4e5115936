"""The allocation-free grouped entry point (iaat_gemm_grouped_noalloc).

Some callers cannot allocate device memory once they are running -- a
serving process that reserved all GPU memory at start-up, for instance, and
treats any later cudaMalloc as a failure because cudaMalloc and cudaFree
synchronise the device and can fail under memory pressure.  For them the
library has one entry point that plans into static host arrays and runs from
a fixed device scratch array.  These tests call it through the C ABI and
check, on two calls in a row, that C equals the FP64 oracle within the
1e-5 / 1e-13 normwise bounds the other tests use, and that it gives the same
C as the regular planned entry point (iaat_plan_create + iaat_gemm_grouped);
that batches with instances cut into pieces work; that a batch whose pieces
exceed the scratch's task limit is refused with nothing enqueued; and that a
capturing stream is refused.  This file is collected last.
"""
import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

from .gpu_util import compare, padding_untouched, to_device
from .test_gemm_gpu import piece_batch

pytestmark = pytest.mark.gpu

TOL = {np.float32: 1e-5, np.float64: 1e-13}


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_09822_gb300 import build
    build.build()
    iaat.lib()
    return torch


def _ddt(dtype):
    return iaat.IAAT_F32 if dtype == np.float32 else iaat.IAAT_F64


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_noalloc_matches_oracle_and_planned_entry_point_twice(cuda, dtype):
    torch = cuda
    b = W.random_small(3000, seed=77, dtype=dtype, max_dim=80, pad_max=3, misalign_max=1)
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    tA, tB, tC, descs = to_device(b)
    C0 = tC.clone()
    s = torch.cuda.current_stream()
    plan = iaat.iaat_plan_create(descs, _ddt(dtype))
    iaat.iaat_gemm_grouped(plan, s)
    iaat.iaat_plan_check(plan, s)
    planned = tC.cpu().numpy()
    plan.destroy()
    for call in range(2):
        tC.copy_(C0)
        iaat.iaat_gemm_grouped_noalloc(descs, _ddt(dtype), s)
        iaat.iaat_plan_check(None, s)
        got = tC.cpu().numpy()
        err = compare(b, got)
        assert not err["nan"], (call, err)
        assert err["eps_batch"] <= TOL[dtype] and err["eps_inst_max"] <= TOL[dtype], (call, err)
        assert padding_untouched(b, got), call
        # the same tiling and kernel as the planned entry point: the same bits
        assert np.array_equal(got.view(np.uint8), planned.view(np.uint8)), call


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_noalloc_instances_cut_into_pieces(cuda, dtype):
    """Instances far beyond one stage on one side (512000 x 1 x 1 and the
    like) are cut into pieces inside the scratch's task limit; integer
    inputs, so the result is exact."""
    torch = cuda
    b = piece_batch(dtype, 15)
    tA, tB, tC, descs = to_device(b)
    s = torch.cuda.current_stream()
    for call in range(2):
        iaat.iaat_gemm_grouped_noalloc(descs, _ddt(dtype), s)
        iaat.iaat_plan_check(None, s)
        got = tC.cpu().numpy()
        tC.copy_(torch.from_numpy(b.C).to(tC.device))
        err = compare(b, got)
        assert err["exact"], (call, err)
        assert padding_untouched(b, got), call


def test_noalloc_rejects_too_many_instances(cuda):
    d = np.zeros(8193, iaat.DESC_DTYPE)
    for k, v in dict(M=1, N=1, K=1, lda=1, ldb=1, ldc=1, alpha=1.0, beta=0.0, A=0x1000, B=0x2000,
                     C=0x3000).items():
        d[k] = v
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_gemm_grouped_noalloc(d, iaat.IAAT_F32)
    assert e.value.status == 1 and "8192" in e.value.message


def test_noalloc_rejects_too_many_pieces_and_enqueues_nothing(cuda):
    """Five instances of 512000 x 1 x 1 need about 2000 pieces each, more than
    the 8192 tasks the scratch holds: the call is refused before anything is
    enqueued, and C keeps its values."""
    torch = cuda
    rng = np.random.default_rng(5)
    b = W.make_batch([512000] * 5, [1] * 5, [1] * 5, [0] * 5, [0] * 5, 1.0, 0.5, np.float32, rng,
                     dist="int")
    tA, tB, tC, descs = to_device(b)
    before = tC.cpu().numpy()
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_gemm_grouped_noalloc(descs, iaat.IAAT_F32, torch.cuda.current_stream())
    assert e.value.status == 1 and "8192" in e.value.message
    torch.cuda.synchronize()
    iaat.iaat_plan_check(None, torch.cuda.current_stream())
    assert np.array_equal(tC.cpu().numpy().view(np.uint8), before.view(np.uint8))


def test_noalloc_refuses_stream_capture(cuda):
    """A capturing stream is refused with IAAT_ERR_UNSUPPORTED: the call
    copies its plan from host arrays the next call reuses, so a captured
    call could not be replayed."""
    torch = cuda
    b = W.random_small(50, seed=3, max_dim=8)
    tA, tB, tC, descs = to_device(b)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(g, stream=s):
        try:
            iaat.iaat_gemm_grouped_noalloc(descs, iaat.IAAT_F32, s)
        except iaat.IaatError as e:
            status = e.status
    assert status == 4
