"""The pack step kept for the ablation (the GPU analogue of Fig. 3): packing
op(A) and op(B) into tight NN copies and running the grouped plan on them
gives the GEMM of the original instances -- the same values as the no-pack
path (each element is the same FMA sequence in k order) and the FP64
oracle within tolerance."""
import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

from .gpu_util import compare, gather_index, padding_untouched, run_grouped, to_device

pytestmark = pytest.mark.gpu

TOL = {np.float32: 1e-5, np.float64: 1e-13}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_09822_gb300 import build
    build.build()
    iaat.lib()
    return torch


def _packed_run(b, torch):
    tA, tB, tC, descs = to_device(b)
    dtype = iaat.IAAT_F32 if b.dtype == np.float32 else iaat.IAAT_F64
    pk = iaat.iaat_pack_create(descs, dtype)
    s = torch.cuda.current_stream()
    iaat.iaat_pack_run(pk, s)
    plan = iaat.iaat_plan_create(pk.packed, dtype)
    iaat.iaat_gemm_grouped(plan, s)
    iaat.iaat_plan_check(plan, s)
    out = tC.cpu().numpy()
    plan.destroy()
    moved = pk.bytes_moved
    packed = pk.packed.copy()
    pk.destroy()
    return out, packed, moved


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_packed_path_equals_the_direct_path(dtype, cuda):
    b = W.random_small(2000, seed=51, dtype=dtype, max_dim=40, pad_max=4, misalign_max=3)
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    C, packed, moved = _packed_run(b, cuda)
    err = compare(b, C)
    assert not err["nan"] and err["eps_batch"] <= TOL[dtype] and err["eps_inst_max"] <= TOL[dtype], err
    assert padding_untouched(b, C)
    D, _ = run_grouped(b)
    gi, _ = gather_index(b, "C")
    assert np.array_equal(C[gi], D[gi])
    assert (packed["transA"] == 0).all() and (packed["transB"] == 0).all()
    used = (b.M > 0) & (b.N > 0) & (b.K > 0) & (b.alpha != 0)
    esz = np.dtype(dtype).itemsize
    M, N, K = (x.astype(np.int64) for x in (b.M, b.N, b.K))
    assert moved == int(2 * esz * np.sum(np.where(used, M * K + K * N, 0)))
    assert (packed["A"][~used] == 0).all()


def test_packed_integers_bit_exact(cuda):
    rng = np.random.default_rng(52)
    n = 1000
    b = W.random_small(n, seed=53, max_dim=24, pad_max=3, dist="int", misalign_max=2,
                       alpha=rng.choice([0.0, 1.0, -1.0, 2.0], n), beta=rng.choice([0.0, 1.0, -1.0, 2.0], n))
    C, _, _ = _packed_run(b, cuda)
    assert compare(b, C)["exact"]
