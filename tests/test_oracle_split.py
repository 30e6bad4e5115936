"""Pins for the emulation oracle of the tensor-core paths (CPU only).

``oracle/split_oracle.py`` rounds the operands the way each tensor-core path
does and adds that path's products in FP64.  Its pieces are pinned to
independent implementations and to the arithmetic: BF16 and FP16 rounding to
torch's conversions, TF32 rounding to a brute-force nearest-even choice, the
splits to their exactness properties, and the emulated GEMMs to the exact
GEMM (equal on integer inputs, within each split's error bound on random
ones).  A planted mistake (a product left out) breaks the bound.
"""
import numpy as np
import pytest

import oracle
from oracle import split_oracle as S
from paper_2208_09822_gb300 import workloads as W

torch = pytest.importorskip("torch")


def _samples(n=200_000, seed=0):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    u[: n // 8] = (u[: n // 8] & 0xFFFF0000) | 0x8000          # BF16 ties
    u[n // 8: n // 4] = (u[n // 8: n // 4] & 0xFFFFE000) | 0x1000   # TF32 ties
    u[n // 4: n // 3] &= 0x807FFFFF                            # subnormals
    x = u.view(np.float32)
    return x[np.isfinite(x)]


def test_bf16_matches_torch():
    x = _samples()
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(S.bf16_rn(x).view(np.uint32), ref.view(np.uint32))


def test_fp16_matches_torch():
    x = _samples(seed=1)
    x = x[np.abs(x) < 60000]
    ref = torch.from_numpy(x).half().float().numpy()
    got = S.fp16_rn(x)
    assert np.array_equal(got, ref) or np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_tf32_is_the_nearest_even_candidate():
    x = _samples(20_000, seed=2)
    u = x.view(np.uint32).astype(np.uint64)
    lo = (u & 0xFFFFE000).astype(np.uint32).view(np.float32).astype(np.float64)
    hi_bits = (u & 0xFFFFE000) + 0x2000
    got = S.tf32_rn(x).view(np.uint32)
    for i in range(len(x)):
        xv = float(x[i])
        a = float(lo[i])
        b = float(np.array([hi_bits[i]], np.uint64).astype(np.uint32).view(np.float32)[0])
        da, db = abs(xv - a), abs(b - xv)
        if da < db or (da == db and ((int(u[i]) >> 13) & 1) == 0):
            want = int(u[i]) & 0xFFFFE000
        else:
            want = int(hi_bits[i]) & 0xFFFFFFFF
        assert int(got[i]) == want, (hex(int(u[i])), hex(int(got[i])), hex(want))


@pytest.mark.parametrize("prec,bound", [("3xbf16", 2.0**-16), ("6xbf16", 2.0**-24)])
def test_splits_are_exact_sums_within_their_bound(prec, bound):
    x = np.random.default_rng(3).standard_normal(100_000).astype(np.float32)
    terms = S.split_terms(x, prec)
    for t in terms:
        assert np.array_equal(S.bf16_rn(t), t)       # every term is a BF16 value
    total = sum(t.astype(np.float64) for t in terms)
    assert np.all(np.abs(total - x) <= bound * np.abs(x.astype(np.float64)) + 1e-45)


def pin_failures(products=None):
    fails = []
    # integer entries: every split term past the first is zero, so each path is the exact GEMM
    rng = np.random.default_rng(4)
    n = 400
    b = W.random_small(n, seed=5, max_dim=12, pad_max=2, dist="int", alpha=rng.choice([0.0, 1.0, -1.0, 2.0], n),
                       beta=rng.choice([0.0, 1.0, -1.0, 2.0], n))
    exact, off = oracle.gemm_batch(b)
    for prec in S.PRECISIONS:
        got, off2 = S.tc_gemm_batch(b, prec, products=products if prec == "3xbf16" else None)
        if not (np.array_equal(off, off2) and np.array_equal(got, exact)):
            fails.append(f"integers-{prec}")
    # random entries: within each split's error bound of the exact GEMM, per instance
    # |C_split - C| <= u_split * |alpha| * (|A| |B|) elementwise
    b = W.random_small(300, seed=6, max_dim=20, pad_max=2)
    exact, off = oracle.gemm_batch(b)
    ubound = {"3xbf16": 2.0**-15, "6xbf16": 2.0**-22, "tf32": 2.0**-10, "fp16": 2.0**-9}
    for prec in S.PRECISIONS:
        got, _ = S.tc_gemm_batch(b, prec, products=products if prec == "3xbf16" else None)
        ok = True
        for t in range(b.count):
            M, N, K = int(b.M[t]), int(b.N[t]), int(b.K[t])
            if M * N == 0 or K == 0:
                continue
            ta, tb = int(b.transA[t]), int(b.transB[t])
            A = S._dense(b.A, b.offA[t], K if ta else M, M if ta else K, int(b.lda[t])).astype(np.float64)
            B = S._dense(b.B, b.offB[t], N if tb else K, K if tb else N, int(b.ldb[t])).astype(np.float64)
            opA = A.T if ta else A
            opB = B.T if tb else B
            lim = ubound[prec] * abs(float(b.alpha[t])) * (np.abs(opA) @ np.abs(opB))
            d = np.abs(got[off[t]:off[t] + M * N] - exact[off[t]:off[t] + M * N]).reshape(N, M).T
            if not np.all(d <= lim + 1e-300):
                ok = False
                break
        if not ok:
            fails.append(f"bound-{prec}")
    return fails


def test_emulated_paths_hold_their_pins():
    assert pin_failures() == []


def test_a_dropped_product_is_caught():
    assert "bound-3xbf16" in pin_failures(products=((0, 0), (1, 0)))
