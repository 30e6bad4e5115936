"""Plans over contiguous instance ranges of one batch reproduce the one-plan
result bit for bit, on every path: each instance's arithmetic is fixed by
its own tiling (CUDA cores) or by its own rows and columns of a tensor-core
pack (the packs' zero padding adds exact zeros), never by its neighbours.
bench.py's end-to-end leg pipelines copies and launches over such ranges,
and a multi-GPU run gives each rank one."""
import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W
from paper_2208_09822_gb300.shard import instance_cost, shard_bounds

from .gpu_util import compare, padding_untouched, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_09822_gb300 import build
    build.build()
    iaat.lib()
    return torch


@pytest.mark.parametrize("prec", [iaat.IAAT_PREC_DEFAULT, iaat.IAAT_PREC_3XBF16, iaat.IAAT_PREC_TF32,
                                  iaat.IAAT_PREC_FP16, iaat.IAAT_PREC_6XBF16])
def test_range_plans_equal_the_whole_plan(cuda, prec):
    torch = cuda
    b = W.uneven(count=20000, seed=21)
    tA, tB, tC, descs = to_device(b)
    C0 = tC.clone()
    s = torch.cuda.current_stream()
    whole = iaat.iaat_plan_create(descs, iaat.IAAT_F32, prec)
    iaat.iaat_gemm_grouped(whole, s)
    iaat.iaat_plan_check(whole, s)
    ref = tC.cpu().numpy()
    whole.destroy()
    tC.copy_(C0)
    ranges = [r for r in shard_bounds(instance_cost(b.M, b.N, b.K, b.beta != 0), 5) if r[1] > r[0]]
    assert len(ranges) == 5 and ranges[0][0] == 0 and ranges[-1][1] == b.count
    for b0, b1 in ranges:
        p = iaat.iaat_plan_create(descs[b0:b1], iaat.IAAT_F32, prec)
        iaat.iaat_gemm_grouped(p, s)
        iaat.iaat_plan_check(p, s)
        p.destroy()
    got = tC.cpu().numpy()
    assert np.array_equal(got, ref)
    assert padding_untouched(b, got)
    if prec in (iaat.IAAT_PREC_DEFAULT, iaat.IAAT_PREC_3XBF16):
        assert compare(b, got)["eps_batch"] <= 1e-5
