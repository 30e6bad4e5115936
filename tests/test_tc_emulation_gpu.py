"""Parity of every tensor-core path with the emulation oracle of its own
arithmetic (``oracle/split_oracle.py``: the path's operand rounding and
products, summed in FP64).  The paths accumulate in FP32, so they must match
it to FP32 accumulation error -- far tighter than their distance from the
exact GEMM (TF32 and FP16 are about 3e-4 from it): eps_batch and the guarded
per-instance error <= 1e-6 (measured: at most 3.4e-7 and 2.8e-7), on the
uneven distribution, small random instances of every case with ld padding
and misaligned starts, and the sweep's shapes with entries scaled by
10^U[-3,3] (FP16 subnormals included)."""
import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

from .gpu_util import errors, padding_untouched, run_grouped

pytestmark = pytest.mark.gpu

PRECS = {"3xbf16": iaat.IAAT_PREC_3XBF16, "tf32": iaat.IAAT_PREC_TF32, "fp16": iaat.IAAT_PREC_FP16,
         "6xbf16": iaat.IAAT_PREC_6XBF16}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_09822_gb300 import build
    build.build()
    iaat.lib()
    return torch


def _batches():
    small = W.random_small(3000, seed=31, max_dim=40, pad_max=3, misalign_max=2)
    small = small.select(np.nonzero(W.in_domain(small.M, small.N, small.K, small.transA, small.transB))[0])
    return {"uneven": W.uneven(count=20000, seed=30), "small": small,
            "scaled": W.sweep_mixed("NN", per_shape=1, seed=32, decades=3)}


@pytest.fixture(scope="module")
def batches():
    return _batches()


@pytest.mark.parametrize("prec", sorted(PRECS))
@pytest.mark.parametrize("which", ["uneven", "small", "scaled"])
def test_tensor_core_paths_match_their_emulation(prec, which, batches):
    from oracle import split_oracle as S
    b = batches[which]
    C, _ = run_grouped(b, PRECS[prec])
    ref, _ = S.tc_gemm_batch(b, prec)
    e = errors(b, C, ref)
    assert not e["nan"]
    assert e["eps_batch"] <= 1e-6 and e["eps_inst_max"] <= 1e-6, e
    assert padding_untouched(b, C)
