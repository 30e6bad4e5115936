"""Parity of the warp-direct CUDA-core kernel (plan option kernel = 4) with
the FP64 oracle: every warp runs its own blocks of at most 32 rows straight
from global memory, its lanes laid out as column groups of the block's rows.
Exact integer cases in FP32 and FP64 and every trans case, the uneven batch
(bit-identical to the stage-program kernel, which sums in the same order),
edge cases, instances cut into blocks, K in several register passes, graph
replay, a corrupted plan, and the routed tensor-core plan with its CUDA-core
part on this kernel."""
import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

from .gpu_util import compare, gather_index, padding_untouched, run_grouped, to_device
from .test_gemm_gpu import piece_batch

pytestmark = pytest.mark.gpu

DIRECT = 4


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_09822_gb300 import build
    build.build()
    iaat.lib()
    return torch


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("max_dim", [6, 40, 80])
def test_integer_inputs_bit_exact(dtype, max_dim):
    """Integer inputs, products and partial sums: the result must equal the
    oracle bit for bit, so the lane layout, the staged op(B) block, the C0
    copies and the epilogue are checked element by element in all four trans
    cases and every K class (one pass of 4, 8, 16, 32 values, and chunks)."""
    rng = np.random.default_rng(80 + max_dim)
    n = 1500 if max_dim < 80 else 400
    b = W.random_small(n, seed=81 + max_dim, max_dim=max_dim, pad_max=3, dist="int", misalign_max=3,
                       alpha=rng.choice([0.0, 1.0, -1.0, 2.0], n), beta=rng.choice([0.0, 1.0, -1.0, 2.0], n),
                       dtype=dtype)
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    C, info = run_grouped(b, kernel=DIRECT)
    assert info["kernel_family"] == 4
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


def test_uneven_batch_matches_the_stage_programs_bit_for_bit():
    """Both kernels sum each dot product in k order with fused multiply-adds
    and write alpha*acc + beta*C0 the same way, so the results are identical;
    and both are within FP32 rounding of the oracle."""
    b = W.uneven(count=40000, seed=47)
    C, info = run_grouped(b, kernel=DIRECT)
    C1, _ = run_grouped(b, kernel=1)
    assert np.array_equal(C, C1)
    err = compare(b, C)
    assert not err["nan"]
    assert err["eps_inst_max"] <= 1e-5, err
    assert padding_untouched(b, C)


def test_fp64_batch():
    rng = np.random.default_rng(3)
    b = W.random_small(3000, seed=33, max_dim=48, pad_max=5, dtype=np.float64,
                       alpha=rng.uniform(-2, 2, 3000), beta=rng.uniform(-2, 2, 3000))
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    C, info = run_grouped(b, kernel=DIRECT)
    C1, _ = run_grouped(b, kernel=1)
    assert np.array_equal(C, C1)
    err = compare(b, C)
    assert err["eps_batch"] <= 1e-13, err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_edge_cases(dtype):
    """Empty sizes, K = 0, alpha = 0 (beta*C0 exactly; C untouched when beta
    is 1), beta = 0 with NaN in C (never read), one row, one column, the
    largest square shape, K at each pass boundary (4, 5, 8, 9, 16, 17, 32,
    33) and one-row blocks of many column groups."""
    rng = np.random.default_rng(23)
    M = [0, 5, 7, 3, 9, 4, 80, 1, 6, 33, 32, 31, 1, 17, 2, 8]
    N = [5, 0, 7, 3, 9, 4, 80, 1, 6, 70, 17, 16, 80, 1, 33, 8]
    K = [3, 3, 0, 4, 9, 4, 80, 1, 5, 17, 33, 16, 32, 8, 4, 33]
    al = [1.0, 1.0, 1.5, 0.0, 1.0, 0.0, 1.0, -2.0, 1.0, 0.5, 1.0, 2.0, 1.0, -1.0, 1.0, 0.5]
    be = [0.5, 0.5, 2.0, 3.0, 0.0, 1.0, 0.0, 0.0, 1.0, -1.0, 0.5, 0.0, 1.0, 2.0, 0.0, 1.0]
    n = len(M)
    ta = [0, 1, 0, 1, 0, 1, 0, 1, 0, 0, 1, 0, 1, 0, 1, 1]
    tb = [0, 0, 1, 1, 0, 0, 0, 1, 1, 1, 0, 1, 0, 1, 1, 0]
    b = W.make_batch(M, N, K, ta, tb, al, be, dtype, rng, pad=rng.integers(0, 3, (n, 3)), dist="int")
    assert W.in_domain(b.M, b.N, b.K, b.transA, b.transB).all()
    for t in np.nonzero(np.asarray(be) == 0)[0]:
        idx = b.offC[t] + np.arange(N[t])[None, :] * b.ldc[t] + np.arange(M[t])[:, None]
        b.C[idx.ravel()] = np.nan
    C, info = run_grouped(b, kernel=DIRECT)
    err = compare(b, C)
    assert not err["nan"], err
    assert err["exact"], err
    assert padding_untouched(b, C)
    for t, scale in ((3, 3.0), (5, 1.0)):
        gi, _ = gather_index(b, "C", np.array([t]))
        assert np.array_equal(C[gi], (b.C[gi] * dtype(scale)).astype(dtype))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_instances_cut_into_blocks(dtype):
    """Instances far beyond one block on one side or both (up to 512000 rows
    or columns), K beyond one register pass: exact."""
    b = piece_batch(dtype, 25)
    C, info = run_grouped(b, kernel=DIRECT)
    assert info["tasks"] > b.count
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_long_k_in_chunks(dtype):
    """1 x 1 x K up to the domain's bound, 32 x 32 x 500 and TN / NT blocks
    of K = 36..480: K runs in register passes, the partial sums kept between
    them; integer entries keep every partial sum exact."""
    rng = np.random.default_rng(6)
    K = [20000, 512000, 40000, 500, 480, 36, 100]
    b = W.make_batch([1, 1, 2, 32, 30, 30, 7], [1, 1, 3, 32, 31, 30, 9], K, [0, 0, 0, 0, 0, 1, 1],
                     [1, 1, 0, 0, 1, 0, 1], [1.0, -0.5, 2.0, 1.0, -1.0, 1.0, 2.0], [0.5, 0.0, 1.0, 0.0, 2.0, -1.0, 0.0],
                     dtype, rng, pad=np.zeros((7, 3), np.int64), dist="int")
    assert W.in_domain(b.M, b.N, b.K, b.transA, b.transB).all()
    C, info = run_grouped(b, kernel=DIRECT)
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


def test_graph_replay(cuda):
    torch = cuda
    b = W.uneven(count=5000, seed=49)
    tA, tB, tC, descs = to_device(b)
    C0 = tC.clone()
    plan = iaat.iaat_plan_create(descs, iaat.IAAT_F32, kernel=DIRECT)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        iaat.iaat_gemm_grouped(plan, s)
    iaat.iaat_plan_check(plan, s)
    first = tC.cpu().numpy()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        iaat.iaat_gemm_grouped(plan, s)
    for _ in range(3):
        tC.copy_(C0)
        with torch.cuda.stream(s):
            g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(tC.cpu().numpy(), first)
    iaat.iaat_plan_check(plan, s)
    assert compare(b, first)["eps_inst_max"] <= 1e-5
    plan.destroy()


def test_injected_fault_is_reported_and_context_survives(cuda):
    torch = cuda
    b = W.random_small(500, seed=10, max_dim=16)
    tA, tB, tC, descs = to_device(b)
    bad = iaat.iaat_plan_create(descs, iaat.IAAT_F32, inject_fault=1, kernel=DIRECT)
    iaat.iaat_gemm_grouped(bad, torch.cuda.current_stream())
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_check(bad, torch.cuda.current_stream())
    assert e.value.status == 6
    bad.destroy()
    C, _ = run_grouped(b, kernel=DIRECT)
    assert compare(b, C)["eps_batch"] <= 1e-5


@pytest.mark.parametrize("mnk", [0, 16 ** 3])
def test_routed_plan_with_the_direct_kernel(mnk):
    """The routed 3xBF16 plan with its CUDA-core part on this kernel: the
    same values as with that part on the stage programs, every instance
    within 1e-5."""
    b = W.uneven(count=40000, seed=51)
    C, info = run_grouped(b, iaat.IAAT_PREC_3XBF16, route_k_below=8, route_mnk_below=mnk, route_kernel=DIRECT)
    assert info["kernels"] == 2
    C1, _ = run_grouped(b, iaat.IAAT_PREC_3XBF16, route_k_below=8, route_mnk_below=mnk, route_kernel=1)
    assert np.array_equal(C, C1)
    err = compare(b, C)
    assert err["eps_inst_max"] <= 1e-5, err
    assert padding_untouched(b, C)
