"""Parity of the warp-tile tensor-core kernel (plan option kernel = 3) with
the FP64 oracle: every warp stages, converts and multiplies its own blocks of
at most 32 x 32 of C, op(A) from tensor memory.  The same checks as for the
other tensor-core kernels: exact integer cases in every precision, the
uneven batch, edge cases, instances cut into blocks, K staged in several
ring items (up to the domain's 1 x 1 x 512000), graph replay, a corrupted
plan and the routed plan."""
import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

from .gpu_util import compare, gather_index, padding_untouched, run_grouped, to_device
from .test_gemm_gpu import piece_batch

pytestmark = pytest.mark.gpu

WARP = 3
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


@pytest.mark.parametrize("prec", sorted(PRECS))
@pytest.mark.parametrize("max_dim", [6, 40, 80])
def test_integer_inputs_bit_exact(prec, max_dim):
    """Every input, product and partial sum is an integer every format holds
    exactly, so each path must equal the oracle bit for bit: the staging,
    the tensor-memory layout of op(A), the B tiles and the epilogue are
    checked element by element, in all four trans cases."""
    rng = np.random.default_rng(70 + max_dim)
    n = 1500 if max_dim < 80 else 400
    b = W.random_small(n, seed=71 + max_dim, max_dim=max_dim, pad_max=3, dist="int", misalign_max=3,
                       alpha=rng.choice([0.0, 1.0, -1.0, 2.0], n), beta=rng.choice([0.0, 1.0, -1.0, 2.0], n))
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    C, info = run_grouped(b, PRECS[prec], kernel=WARP)
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("prec", ["3xbf16", "6xbf16", "tf32", "fp16"])
def test_uneven_batch(prec):
    b = W.uneven(count=40000, seed=41)
    C, info = run_grouped(b, PRECS[prec], kernel=WARP)
    err = compare(b, C)
    assert not err["nan"]
    tol = {"3xbf16": 1e-5, "6xbf16": 1e-5, "tf32": 1e-3, "fp16": 1e-3}[prec]
    assert err["eps_batch"] <= tol, err
    if prec == "6xbf16":
        assert err["eps_inst_max"] <= 1e-5, err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("prec", sorted(PRECS))
def test_edge_cases(prec):
    """Empty sizes, K = 0, alpha = 0 (beta*C0 exactly; C untouched when beta
    is 1), beta = 0 with NaN in C (never read), the largest square shape,
    blocks of 17..32 columns (MMA N = 32) and of up to 16 (N = 16)."""
    rng = np.random.default_rng(19)
    M = [0, 5, 7, 3, 9, 4, 80, 1, 6, 33, 32, 31]
    N = [5, 0, 7, 3, 9, 4, 80, 1, 6, 70, 17, 16]
    K = [3, 3, 0, 4, 9, 4, 80, 1, 6, 17, 33, 15]
    al = [1.0, 1.0, 1.5, 0.0, 1.0, 0.0, 1.0, -2.0, 1.0, 0.5, 1.0, 2.0]
    be = [0.5, 0.5, 2.0, 3.0, 0.0, 1.0, 0.0, 0.0, 1.0, -1.0, 0.5, 0.0]
    n = len(M)
    ta = [0, 1, 0, 1, 0, 1, 0, 1, 0, 0, 1, 0]
    tb = [0, 0, 1, 1, 0, 0, 0, 1, 1, 1, 0, 1]
    b = W.make_batch(M, N, K, ta, tb, al, be, np.float32, rng, pad=rng.integers(0, 3, (n, 3)), dist="int")
    for t in np.nonzero(np.asarray(be) == 0)[0]:
        idx = b.offC[t] + np.arange(N[t])[None, :] * b.ldc[t] + np.arange(M[t])[:, None]
        b.C[idx.ravel()] = np.nan
    C, info = run_grouped(b, PRECS[prec], kernel=WARP)
    err = compare(b, C)
    assert not err["nan"], err
    assert err["exact"], err
    assert padding_untouched(b, C)
    for t, scale in ((3, 3.0), (5, 1.0)):
        gi, _ = gather_index(b, "C", np.array([t]))
        assert np.array_equal(C[gi], (b.C[gi] * np.float32(scale)).astype(np.float32))


@pytest.mark.parametrize("prec", ["3xbf16", "tf32"])
def test_instances_cut_into_blocks(prec):
    """Instances small by MNK but far beyond one 32 x 32 block on one side:
    cut into blocks, integer inputs, exact."""
    b = piece_batch(np.float32, 24)
    C, info = run_grouped(b, PRECS[prec], kernel=WARP)
    assert info["tasks"] > b.count
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("prec", ["3xbf16", "tf32"])
def test_long_k_in_several_items(prec):
    """1 x 1 x K up to the domain's bound, 32 x 32 x 500 and a TN block of
    K = 36: K staged in several ring items, accumulated across them; integer
    entries keep every partial sum exact."""
    rng = np.random.default_rng(5)
    K = [20000, 512000, 40000, 500, 480, 36]
    b = W.make_batch([1, 1, 2, 32, 30, 30], [1, 1, 3, 32, 31, 30], K, [0, 0, 0, 0, 0, 1], [1, 1, 0, 0, 1, 0],
                     [1.0, -0.5, 2.0, 1.0, -1.0, 1.0], [0.5, 0.0, 1.0, 0.0, 2.0, -1.0], np.float32, rng,
                     pad=np.zeros((6, 3), np.int64), dist="int")
    assert W.in_domain(b.M, b.N, b.K, b.transA, b.transB).all()
    C, info = run_grouped(b, PRECS[prec], kernel=WARP)
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


def test_graph_replay(cuda):
    torch = cuda
    b = W.uneven(count=5000, seed=43)
    tA, tB, tC, descs = to_device(b)
    C0 = tC.clone()
    plan = iaat.iaat_plan_create(descs, iaat.IAAT_F32, iaat.IAAT_PREC_3XBF16, kernel=WARP)
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
    assert compare(b, first)["eps_batch"] <= 1e-5
    plan.destroy()


def test_injected_fault_is_reported_and_context_survives(cuda):
    torch = cuda
    b = W.random_small(500, seed=9, max_dim=16)
    tA, tB, tC, descs = to_device(b)
    bad = iaat.iaat_plan_create(descs, iaat.IAAT_F32, iaat.IAAT_PREC_3XBF16, inject_fault=1, kernel=WARP)
    iaat.iaat_gemm_grouped(bad, torch.cuda.current_stream())
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_check(bad, torch.cuda.current_stream())
    assert e.value.status == 6
    bad.destroy()
    C, _ = run_grouped(b, iaat.IAAT_PREC_3XBF16, kernel=WARP)
    assert compare(b, C)["eps_batch"] <= 1e-5


def test_routed_plan_meets_the_per_instance_bound():
    """K < 8 routed to the FP32 CUDA-core kernel (its default plan), the rest
    on the warp-tile kernel: every instance within 1e-5."""
    b = W.uneven(count=40000, seed=45)
    C, info = run_grouped(b, iaat.IAAT_PREC_3XBF16, kernel=WARP, route_k_below=8)
    assert info["kernels"] == 2
    err = compare(b, C)
    assert err["eps_inst_max"] <= 1e-5, err
    assert padding_untouched(b, C)
