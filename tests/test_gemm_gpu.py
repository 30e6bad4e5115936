"""Parity of the CUDA path with the FP64 oracle (GB300).

Tolerances (from the build's target): normwise relative error over a batch
eps_batch <= 1e-5 for FP32 and <= 1e-13 for FP64; the per-instance guarded
error (each instance normalised by |alpha| |A| |B| + |beta| |C0|) is held to
the same bounds.  Integer-valued inputs, whose every partial sum is exact in
either type, must match bit for bit.
"""
import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

from .gpu_util import compare, padding_untouched, run_grouped, to_device

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


def _assert_ok(batch, C, err, tol):
    assert not err["nan"]
    assert err["eps_batch"] <= tol, err
    assert err["eps_inst_max"] <= tol, err
    assert padding_untouched(batch, C)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("seed", [21, 22])
def test_random_small_every_case(dtype, seed):
    b = W.random_small(3000, seed=seed, dtype=dtype, max_dim=24, pad_max=5, misalign_max=3)
    C, info = run_grouped(b)
    _assert_ok(b, C, compare(b, C), TOL[dtype])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_integer_inputs_bit_exact(dtype):
    rng = np.random.default_rng(3)
    n = 1500
    b = W.random_small(n, seed=4, dtype=dtype, max_dim=20, pad_max=3, dist="int",
                       misalign_max=2, alpha=rng.choice([0.0, 1.0, -1.0, 2.0], n),
                       beta=rng.choice([0.0, 1.0, -1.0, 2.0], n))
    C, _ = run_grouped(b)
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


def test_uniform16_full():
    b = W.uniform16()
    C, info = run_grouped(b)
    assert info["active"] == 10000
    _assert_ok(b, C, compare(b, C), 1e-5)


@pytest.mark.parametrize("case", ["NN", "NT", "TN", "TT"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_sweep_every_shape(case, dtype):
    b = W.sweep_mixed(case, dtype=dtype, per_shape=2)
    C, _ = run_grouped(b)
    _assert_ok(b, C, compare(b, C), TOL[dtype])


def test_uneven_batch_full():
    b = W.uneven()
    C, info = run_grouped(b)
    assert info["active"] == b.count
    err = compare(b, C)
    _assert_ok(b, C, err, 1e-5)


def test_fc64_batch_full():
    b = W.fc64()
    C, info = run_grouped(b)
    err = compare(b, C)
    _assert_ok(b, C, err, 1e-13)


@pytest.mark.parametrize("case,shape", [("NN", (80, 80, 80)), ("TN", (32, 32, 32)), ("NT", (1, 1, 1)),
                                        ("TT", (80, 1, 80)), ("NN", (5, 80, 7))])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_sweep_full_launch_sampled(case, shape, dtype):
    """The full 4096-instance launch; a sample of instances checked."""
    b = W.sweep(case, shape, dtype=dtype, count=4096)
    C, _ = run_grouped(b)
    idx = np.random.default_rng(0).choice(b.count, 96, replace=False)
    err = compare(b, C, idx)
    assert err["eps_batch"] <= TOL[dtype] and err["eps_inst_max"] <= TOL[dtype], err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_edge_cases(dtype):
    rng = np.random.default_rng(9)
    M = [0, 5, 7, 3, 9, 4, 80, 1, 6]
    N = [5, 0, 7, 3, 9, 4, 80, 1, 6]
    K = [3, 3, 0, 4, 9, 4, 80, 1, 6]
    al = [1.0, 1.0, 1.5, 0.0, 1.0, 0.0, 1.0, -2.0, 1.0]
    be = [0.5, 0.5, 2.0, 3.0, 0.0, 1.0, 0.0, 0.0, 1.0]
    n = len(M)
    ta = [0, 1, 0, 1, 0, 1, 0, 1, 0]
    tb = [0, 0, 1, 1, 0, 0, 0, 1, 1]
    b = W.make_batch(M, N, K, ta, tb, al, be, dtype, rng, pad=rng.integers(0, 3, (n, 3)))
    # beta == 0 must not read C: put NaN there
    for t in np.nonzero(np.asarray(be) == 0)[0]:
        idx = b.offC[t] + np.arange(N[t])[None, :] * b.ldc[t] + np.arange(M[t])[:, None]
        b.C[idx.ravel()] = np.nan
    C, info = run_grouped(b)
    err = compare(b, C)
    assert not err["nan"], err
    assert err["eps_batch"] <= TOL[dtype]
    assert padding_untouched(b, C)
    # alpha == 0 (instance 3) is exactly beta*C0; alpha == 0, beta == 1 (5) untouched
    from .gpu_util import gather_index
    for t, scale in ((3, 3.0), (5, 1.0)):
        gi, _ = gather_index(b, "C", np.array([t]))
        assert np.array_equal(C[gi], (b.C[gi] * dtype(scale)).astype(dtype))


# Small by MNK, but with one side far beyond a warp block or a stage: the
# planner cuts such instances into row and column pieces (Sec. I bounds
# cbrt(MNK), not the single sizes).
PIECE_SHAPES = [  # M, N, K, transA, transB
    (2000, 256, 1, 0, 0), (512000, 1, 1, 0, 0), (1, 512000, 1, 0, 1), (300, 300, 5, 1, 1),
    (129, 129, 30, 0, 1), (32768, 1, 1, 1, 0), (130, 70, 40, 0, 0), (70, 200, 36, 0, 1),
]


def piece_batch(dtype, seed):
    rng = np.random.default_rng(seed)
    M, N, K, ta, tb = (list(x) for x in zip(*PIECE_SHAPES))
    n = len(M)
    be = [0.5, 0.0, -1.0, 0.5, 2.0, 0.0, 1.0, 0.5]
    b = W.make_batch(M, N, K, ta, tb, [1.5, 1.0, -2.0, 1.0, 0.5, 1.0, 1.0, -1.0], be, dtype, rng,
                     pad=rng.integers(0, 3, (n, 3)), dist="int")
    assert W.in_domain(b.M, b.N, b.K, b.transA, b.transB).all()
    return b


@pytest.mark.parametrize("dtype,kernel", [(np.float32, 0), (np.float32, 1), (np.float64, 0)])
def test_instances_cut_into_pieces(dtype, kernel):
    """Instances beyond one stage: on the stage programs (kernel 1, and FP64)
    cut into row / column pieces; a default FP32 plan sends them to the
    warp-stream kernel, which streams K.  Integer inputs, exact."""
    b = piece_batch(dtype, 14)
    C, info = run_grouped(b, kernel=kernel)
    assert info["tasks"] > b.count
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_large_leading_dimensions(dtype):
    """ld far above the rows: operands are staged column by column."""
    rng = np.random.default_rng(12)
    n = 200
    b = W.make_batch(rng.integers(1, 40, n), rng.integers(1, 40, n), rng.integers(1, 40, n),
                     rng.integers(0, 2, n), rng.integers(0, 2, n), 1.0, 0.5, dtype, rng,
                     pad=rng.integers(100, 300, (n, 3)))
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    C, _ = run_grouped(b)
    _assert_ok(b, C, compare(b, C), TOL[dtype])


@pytest.mark.parametrize("variant", range(1, 6))
def test_every_fp32_variant(variant):
    b = W.random_small(600, seed=100 + variant, dtype=np.float32, max_dim=70, pad_max=4, misalign_max=3)
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    C, _ = run_grouped(b, force_variant=variant)
    _assert_ok(b, C, compare(b, C), 1e-5)


@pytest.mark.parametrize("variant", range(1, 11))
def test_every_fp64_variant(variant):
    b = W.random_small(400, seed=200 + variant, dtype=np.float64, max_dim=70, pad_max=4, misalign_max=1)
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    C, _ = run_grouped(b, force_variant=variant)
    _assert_ok(b, C, compare(b, C), 1e-13)


def test_cuda_graph_replay(cuda):
    torch = cuda
    b = W.random_small(2000, seed=5, max_dim=40, pad_max=3, beta=np.zeros(2000))
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    tA, tB, tC, descs = to_device(b)
    plan = iaat.iaat_plan_create(descs, iaat.IAAT_F32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        iaat.iaat_gemm_grouped(plan, s)   # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        iaat.iaat_gemm_grouped(plan, s)
    tC.fill_(W.C_SENTINEL)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    iaat.iaat_plan_check(plan, s)
    C = tC.cpu().numpy()
    err = compare(b, C)
    assert err["eps_batch"] <= 1e-5 and err["eps_inst_max"] <= 1e-5, err
    plan.destroy()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_single_call(cuda, dtype):
    torch = cuda
    rng = np.random.default_rng(31)
    # the last two need more pieces than one launch's parameter block holds
    # (32): the call takes several launches on the stream
    shapes = [(1, 1, 1, 0, 0), (17, 23, 9, 1, 0), (80, 80, 80, 0, 0), (32, 32, 32, 1, 0),
              (80, 3, 80, 1, 1), (64, 80, 80, 0, 1), (33, 65, 40, 0, 0), (200, 200, 12, 1, 1),
              (5000, 100, 1, 0, 1), (512000, 1, 1, 0, 0), (1, 512000, 1, 0, 1)]
    for M, N, K, ta, tb in shapes:
        b = W.make_batch([M], [N], [K], [ta], [tb], 0.75, -1.25, dtype, rng, pad=[[1, 2, 3]])
        tA, tB, tC, descs = to_device(b)
        d = descs[0]
        fn = iaat.iaat_sgemm if dtype == np.float32 else iaat.iaat_dgemm
        fn(ta, tb, M, N, K, 0.75, int(d["A"]), int(d["lda"]), int(d["B"]), int(d["ldb"]), -1.25,
           int(d["C"]), int(d["ldc"]), torch.cuda.current_stream())
        iaat.iaat_plan_check(None, torch.cuda.current_stream())
        C = tC.cpu().numpy()
        err = compare(b, C)
        assert err["eps_inst_max"] <= TOL[dtype], (M, N, K, err)
        assert padding_untouched(b, C)


def test_injected_fault_is_reported_and_context_survives(cuda):
    torch = cuda
    b = W.random_small(500, seed=7, max_dim=16)
    tA, tB, tC, descs = to_device(b)
    bad = iaat.iaat_plan_create(descs, iaat.IAAT_F32, inject_fault=1)
    iaat.iaat_gemm_grouped(bad, torch.cuda.current_stream())
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_check(bad, torch.cuda.current_stream())
    assert e.value.status == 6
    bad.destroy()
    # the context still works
    C, _ = run_grouped(b)
    assert compare(b, C)["eps_batch"] <= 1e-5


def test_fp64_mixed_tiling_exact():
    """FP64 instances shaped like the fc64 batch (M in {32, 64}, N and K up
    to 80): where the cost model prefers it, C is cut into an exact multiple
    of a wide block and a remainder, each with its own register-tile variant
    (mixed-shape tiling, Sec. V-A); some instances here are cut that way.
    Integer inputs, so the result is exact."""
    rng = np.random.default_rng(41)
    n = 300
    M = rng.choice(np.array([32, 64]), n)
    N = rng.integers(8, 81, n)
    K = rng.integers(8, 81, n)
    b = W.make_batch(M, N, K, rng.integers(0, 2, n) * 0, rng.integers(0, 2, n), rng.choice([1.0, -1.0], n),
                     rng.choice([0.0, 1.0], n), np.float64, rng, pad=rng.integers(0, 4, (n, 3)), dist="int")
    assert W.in_domain(b.M, b.N, b.K, b.transA, b.transB).all()
    C, info = run_grouped(b)
    assert info["tasks"] > info["active"], info
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


def test_ffma_instances_beyond_a_stage_go_to_the_warp_stream_kernel():
    """A default FP32 plan keeps the instances a stage holds whole on the
    stage programs and sends the others (80^3 here) to the warp-stream
    kernel, which streams K: two launches, each part bit for bit what its
    own kernel's plan gives, the whole within the FP32 bound."""
    rng = np.random.default_rng(43)
    n = 600
    big = rng.random(n) < 0.25
    M = np.where(big, 80, rng.integers(1, 33, n))
    N = np.where(big, 80, rng.integers(1, 33, n))
    K = np.where(big, 80, rng.integers(1, 33, n))
    b = W.make_batch(M, N, K, rng.integers(0, 2, n) * 0, rng.integers(0, 2, n), rng.uniform(-2, 2, n),
                     rng.uniform(-2, 2, n), np.float32, rng, pad=rng.integers(0, 4, (n, 3)))
    assert W.in_domain(b.M, b.N, b.K, b.transA, b.transB).all()
    C, info = run_grouped(b)
    assert info["kernels"] == 2 and info["kernel_family"] == 1
    err = compare(b, C)
    assert err["eps_batch"] <= 1e-5 and err["eps_inst_max"] <= 1e-5, err
    assert padding_untouched(b, C)
    from .gpu_util import gather_index
    for kernel, idx in ((1, np.nonzero(~big)[0]), (2, np.nonzero(big)[0])):
        ref, _ = run_grouped(b, kernel=kernel)
        gi, _ = gather_index(b, "C", idx)
        assert np.array_equal(C[gi].view(np.uint32), ref[gi].view(np.uint32)), kernel
