"""Parity of the stream kernels (plan option kernel = 2) with the FP64 oracle:
the CUDA-core warp-stream kernel (every warp streams its own warp tasks) and
the tensor-core pack-stream kernel (four warp groups with a producer warp
each, dense 128-row packs).  The default plans run the stage-program
kernels, which the other GPU test files cover; these are the same checks on
the stream kernels: exact integer cases, the uneven batch, edge cases,
instances cut into pieces, K longer than any pipeline stage (the warp-stream
kernel streams K), graph replay and a corrupted plan."""
import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

from .gpu_util import compare, gather_index, padding_untouched, run_grouped, to_device
from .test_gemm_gpu import piece_batch

pytestmark = pytest.mark.gpu

STREAM = 2
PRECS = {"ffma": iaat.IAAT_PREC_DEFAULT, "3xbf16": iaat.IAAT_PREC_3XBF16, "tf32": iaat.IAAT_PREC_TF32,
         "fp16": iaat.IAAT_PREC_FP16, "6xbf16": iaat.IAAT_PREC_6XBF16}


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
@pytest.mark.parametrize("max_dim", [6, 40])
def test_integer_inputs_bit_exact(prec, max_dim):
    """Every input, product and partial sum is an integer every format holds
    exactly, so each path must equal the oracle bit for bit."""
    rng = np.random.default_rng(50 + max_dim)
    n = 1500
    b = W.random_small(n, seed=51 + max_dim, max_dim=max_dim, pad_max=3, dist="int", misalign_max=3,
                       alpha=rng.choice([0.0, 1.0, -1.0, 2.0], n), beta=rng.choice([0.0, 1.0, -1.0, 2.0], n))
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    C, info = run_grouped(b, PRECS[prec], kernel=STREAM)
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("prec", ["ffma", "3xbf16", "6xbf16"])
def test_uneven_batch(prec):
    b = W.uneven(count=40000, seed=31)
    C, info = run_grouped(b, PRECS[prec], kernel=STREAM)
    err = compare(b, C)
    assert not err["nan"]
    assert err["eps_batch"] <= 1e-5, err
    if prec != "3xbf16":   # 3xBF16 drops Al*Bl, visible per instance at tiny K
        assert err["eps_inst_max"] <= 1e-5, err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("prec", sorted(PRECS))
def test_edge_cases(prec):
    """Empty sizes, K = 0, alpha = 0 (beta*C0 exactly; C untouched when beta
    is 1), beta = 0 with NaN in C (never read), the largest square shape."""
    rng = np.random.default_rng(9)
    M = [0, 5, 7, 3, 9, 4, 80, 1, 6, 33]
    N = [5, 0, 7, 3, 9, 4, 80, 1, 6, 70]
    K = [3, 3, 0, 4, 9, 4, 80, 1, 6, 17]
    al = [1.0, 1.0, 1.5, 0.0, 1.0, 0.0, 1.0, -2.0, 1.0, 0.5]
    be = [0.5, 0.5, 2.0, 3.0, 0.0, 1.0, 0.0, 0.0, 1.0, -1.0]
    n = len(M)
    ta = [0, 1, 0, 1, 0, 1, 0, 1, 0, 0]
    tb = [0, 0, 1, 1, 0, 0, 0, 1, 1, 1]
    b = W.make_batch(M, N, K, ta, tb, al, be, np.float32, rng, pad=rng.integers(0, 3, (n, 3)), dist="int")
    for t in np.nonzero(np.asarray(be) == 0)[0]:
        idx = b.offC[t] + np.arange(N[t])[None, :] * b.ldc[t] + np.arange(M[t])[:, None]
        b.C[idx.ravel()] = np.nan
    C, info = run_grouped(b, PRECS[prec], kernel=STREAM)
    err = compare(b, C)
    assert not err["nan"], err
    assert err["exact"], err
    assert padding_untouched(b, C)
    for t, scale in ((3, 3.0), (5, 1.0)):
        gi, _ = gather_index(b, "C", np.array([t]))
        assert np.array_equal(C[gi], (b.C[gi] * np.float32(scale)).astype(np.float32))


@pytest.mark.parametrize("prec", ["ffma", "3xbf16"])
def test_instances_cut_into_pieces(prec):
    """Instances small by MNK but far beyond one warp block or MMA tile on
    one side: cut into blocks or pieces, integer inputs, exact."""
    b = piece_batch(np.float32, 14)
    C, info = run_grouped(b, PRECS[prec], kernel=STREAM)
    assert info["tasks"] > b.count
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


def test_warp_stream_long_k():
    """1 x 1 x K up to the domain's bound: the stage-program kernels reject
    it (a row of A and a column of B that long do not fit one stage); the
    warp-stream kernel streams K in chunks and computes it."""
    rng = np.random.default_rng(3)
    K = [20000, 512000, 40000]
    # integer entries: every partial sum stays below 2**24, so FP32 is exact
    b = W.make_batch([1, 1, 2], [1, 1, 3], K, [0, 0, 0], [1, 1, 0], [1.0, -0.5, 2.0], [0.5, 0.0, 1.0],
                     np.float32, rng, pad=np.zeros((3, 3), np.int64), dist="int")
    assert W.in_domain(b.M, b.N, b.K, b.transA, b.transB).all()
    C, info = run_grouped(b, iaat.IAAT_PREC_DEFAULT, kernel=STREAM)
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("prec", ["ffma", "3xbf16"])
def test_graph_replay(cuda, prec):
    """Captured in a CUDA graph and replayed: the plan's launch reads only
    device memory the plan owns, so a replay reproduces the first result."""
    torch = cuda
    b = W.uneven(count=5000, seed=33)
    tA, tB, tC, descs = to_device(b)
    C0 = tC.clone()
    plan = iaat.iaat_plan_create(descs, iaat.IAAT_F32, PRECS[prec], kernel=STREAM)
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


@pytest.mark.parametrize("prec", ["ffma", "3xbf16"])
def test_injected_fault_is_reported_and_context_survives(cuda, prec):
    """A corrupted plan (a task record or pack header the kernel must
    refuse) is reported as a device error by iaat_plan_check, and the
    context keeps working."""
    torch = cuda
    b = W.random_small(500, seed=7, max_dim=16)
    tA, tB, tC, descs = to_device(b)
    bad = iaat.iaat_plan_create(descs, iaat.IAAT_F32, PRECS[prec], inject_fault=1, kernel=STREAM)
    iaat.iaat_gemm_grouped(bad, torch.cuda.current_stream())
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_check(bad, torch.cuda.current_stream())
    assert e.value.status == 6
    bad.destroy()
    C, _ = run_grouped(b, PRECS[prec], kernel=STREAM)
    assert compare(b, C)["eps_batch"] <= 1e-5
