"""Parity of the complex CUDA path (CGEMM / ZGEMM, Table I rows 3-4) with the
FP64 complex oracle (GB300).

Tolerances as for the real types: eps_batch and the per-instance guarded
error <= 1e-5 for complex float (FFMA) and <= 1e-13 for complex double
(DFMA).  Gaussian-integer inputs, whose every partial sum is exact in either
component type, must match bit for bit.
"""
import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

from .gpu_util import compare, padding_untouched, plan_for, run_grouped, to_device

pytestmark = pytest.mark.gpu

TOL = {np.complex64: 1e-5, np.complex128: 1e-13}
CTYPES = [np.complex64, np.complex128]


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


@pytest.mark.parametrize("dtype", CTYPES)
@pytest.mark.parametrize("seed", [31, 32])
def test_random_small_every_case(dtype, seed):
    """All four cases, sizes 0..24, ld padding, starts moved by whole
    elements (complex float: 8 bytes past a 16-byte boundary)."""
    b = W.random_small(2500, seed=seed, dtype=dtype, max_dim=24, pad_max=5, misalign_max=3)
    C, info = run_grouped(b)
    _assert_ok(b, C, compare(b, C), TOL[dtype])
    assert info["dtype"] == (iaat.IAAT_C32 if dtype == np.complex64 else iaat.IAAT_C64)
    assert info["flops"] == b.flops()   # Eq. 2: 8*M*N*K per instance


@pytest.mark.parametrize("dtype", CTYPES)
def test_gaussian_integers_bit_exact(dtype):
    rng = np.random.default_rng(33)
    n = 1200
    choices = np.array([0, 1, -1, 1j, 1 + 1j, 2 - 1j])
    b = W.random_small(n, seed=34, dtype=dtype, max_dim=20, pad_max=3, dist="int", misalign_max=2,
                       alpha=choices[rng.integers(0, len(choices), n)],
                       beta=choices[rng.integers(0, len(choices), n)])
    C, _ = run_grouped(b)
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)


@pytest.mark.parametrize("dtype", CTYPES)
@pytest.mark.parametrize("case", ["NN", "NT", "TN", "TT"])
def test_sweep_shapes(dtype, case):
    """Every in-domain shape of the sweep sizes {1,...,80}^3, two instances
    each (the paper's M = N = K sweep and its off-diagonal shapes)."""
    b = W.sweep_mixed(case, dtype=dtype, per_shape=1, seed=35)
    C, _ = run_grouped(b)
    _assert_ok(b, C, compare(b, C), TOL[dtype])


@pytest.mark.parametrize("dtype", CTYPES)
def test_beta_zero_ignores_nan_and_alpha_zero_scales_c(dtype):
    n = 600
    b = W.random_small(n, seed=36, dtype=dtype, max_dim=16, beta=np.zeros(n))
    b.C[:] = complex(np.nan, np.nan)
    C, _ = run_grouped(b)
    err = compare(b, C)
    assert not err["nan"] and err["eps_batch"] <= TOL[dtype]
    b2 = W.random_small(n, seed=37, dtype=dtype, max_dim=16, alpha=np.zeros(n))
    C2, _ = run_grouped(b2)
    _assert_ok(b2, C2, compare(b2, C2), TOL[dtype])


@pytest.mark.parametrize("dtype,variant", [(np.complex64, v) for v in range(1, 6)]
                         + [(np.complex128, v) for v in range(1, 12)])
def test_every_register_tile(dtype, variant):
    b = W.random_small(400, seed=38 + variant, dtype=dtype, max_dim=40, pad_max=2, misalign_max=1)
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    C, _ = run_grouped(b, force_variant=variant)
    _assert_ok(b, C, compare(b, C), TOL[dtype])


@pytest.mark.parametrize("dtype", CTYPES)
def test_large_instances_are_cut_into_pieces(dtype):
    """80^3 complex double operands (300 KB) exceed a pipeline stage, so the
    planner cuts C into pieces; long-K rows and columns too."""
    shapes = [(80, 80, 80), (64, 80, 100), (80, 64, 90), (1, 1, 600), (2, 200, 600), (200, 2, 600)]
    M, N, K = (np.array([s[i] for s in shapes] * 3) for i in range(3))
    n = len(M)
    rng = np.random.default_rng(39)
    ta = np.zeros(n, np.int64)   # NN and NT: TN is bounded by 32^3
    tb = rng.integers(0, 2, n)
    alpha = rng.uniform(-2, 2, n) + 1j * rng.uniform(-2, 2, n)
    beta = rng.uniform(-2, 2, n) + 1j * rng.uniform(-2, 2, n)
    b = W.make_batch(M, N, K, ta, tb, alpha, beta, dtype, rng, pad=rng.integers(0, 4, (n, 3)))
    C, info = run_grouped(b)
    _assert_ok(b, C, compare(b, C), TOL[dtype])
    assert info["tasks"] > info["active"]


@pytest.mark.parametrize("dtype", CTYPES)
def test_uneven_complex_batch_sampled(dtype):
    """The uneven complex batch at full size (100,000 instances, the
    benchmark's launch) checked on every 25th instance."""
    b = W.uneven_complex(100_000, dtype=dtype)
    C, info = run_grouped(b)
    idx = np.arange(0, b.count, 25)
    err = compare(b, C, idx)
    assert not err["nan"]
    assert err["eps_batch"] <= TOL[dtype], err
    assert err["eps_inst_max"] <= TOL[dtype], err
    assert info["flops"] == b.flops()


@pytest.mark.parametrize("dtype", CTYPES)
def test_graph_replay_matches_first_launch(dtype, cuda):
    torch = cuda
    b = W.random_small(800, seed=40, dtype=dtype, max_dim=30, pad_max=2)
    tA, tB, tC, descs = to_device(b)
    C0 = tC.clone()
    plan = plan_for(b, descs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        iaat.iaat_gemm_grouped(plan, s)
    iaat.iaat_plan_check(plan, s)
    first = tC.cpu().numpy()
    tC.copy_(C0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        iaat.iaat_gemm_grouped(plan, s)
    tC.copy_(C0)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g.replay()
    iaat.iaat_plan_check(plan, s)
    assert np.array_equal(tC.cpu().numpy().view(np.uint8), first.view(np.uint8))
    plan.destroy()


def test_corrupt_program_is_reported(cuda):
    """A stage program claiming too many tasks is refused by the producer;
    the bounded waits end and iaat_plan_check reports the error."""
    torch = cuda
    b = W.random_small(200, seed=41, dtype=np.complex64, max_dim=12)
    tA, tB, tC, descs = to_device(b)
    plan = plan_for(b, descs, inject_fault=1)
    s = torch.cuda.current_stream()
    iaat.iaat_gemm_grouped(plan, s)
    with pytest.raises(iaat.IaatError) as e:
        iaat.iaat_plan_check(plan, s)
    assert e.value.status == 6
    plan.destroy()


@pytest.mark.parametrize("dtype", CTYPES)
def test_single_calls(dtype, cuda):
    """iaat_cgemm / iaat_zgemm, one instance per call on one stream, over
    every case and sizes up to the domain's edges (80^3, 1 x 6400 x 80)."""
    torch = cuda
    rng = np.random.default_rng(42)
    shapes = [(1, 1, 1), (3, 5, 2), (16, 16, 16), (33, 17, 9), (80, 80, 80), (1, 6400, 80), (64, 1, 80),
              (32, 32, 32), (20, 30, 0)]
    M, N, K, ta, tb = [], [], [], [], []
    for (m, n, k) in shapes:
        for t in range(4):
            a, b_ = t >> 1, t & 1
            if W.in_domain(m, n, k, a, b_):
                M.append(m); N.append(n); K.append(k); ta.append(a); tb.append(b_)
    n_ = len(M)
    alpha = rng.uniform(-2, 2, n_) + 1j * rng.uniform(-2, 2, n_)
    beta = rng.uniform(-2, 2, n_) + 1j * rng.uniform(-2, 2, n_)
    beta[::5] = 0
    b = W.make_batch(M, N, K, ta, tb, alpha, beta, dtype, rng, pad=rng.integers(0, 3, (n_, 3)))
    tA, tB, tC, descs = to_device(b)
    s = torch.cuda.current_stream()
    call = iaat.iaat_cgemm if dtype == np.complex64 else iaat.iaat_zgemm
    for d, al, be in zip(descs, b.alpha, b.beta):
        call(int(d["transA"]), int(d["transB"]), int(d["M"]), int(d["N"]), int(d["K"]), complex(al), int(d["A"]),
             int(d["lda"]), int(d["B"]), int(d["ldb"]), complex(be), int(d["C"]), int(d["ldc"]), s)
    iaat.iaat_plan_check(None, s)
    C = tC.cpu().numpy()
    _assert_ok(b, C, compare(b, C), TOL[dtype])


def test_zgemm_mixed_tiling_exact():
    """ZGEMM instances whose C the planner cuts into an exact multiple of a
    block and a remainder, each with its own register tile (mixed-shape
    tiling for the DFMA-bound types); Gaussian-integer inputs, so every
    path is exact."""
    rng = np.random.default_rng(57)
    n = 400
    M = rng.integers(1, 81, n)
    N = rng.integers(1, 81, n)
    K = rng.integers(1, 41, n)
    b = W.make_batch(M, N, K, rng.integers(0, 2, n) * 0, rng.integers(0, 2, n), np.ones(n, complex),
                     np.zeros(n, complex), np.complex128, rng, pad=rng.integers(0, 3, (n, 3)), dist="int")
    b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])
    C, info = run_grouped(b)
    assert info["tasks"] > info["active"], info
    err = compare(b, C)
    assert err["exact"], err
    assert padding_untouched(b, C)
