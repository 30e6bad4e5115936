"""Pins for the complex (CGEMM / ZGEMM) oracle (CPU only).

The complex oracle computes the GEMM of Sec. I on the complex types of
Table I (rows 3-4): C = alpha*op(A)*op(B) + beta*C with complex entries and
scalars, op = N or T (no conjugation), column-major.  Each test pins it to
something other than itself:

* numpy's complex128 matmul (a library routine);
* the real oracle, itself pinned in test_oracle_gemm.py: the real and
  imaginary parts of op(A)op(B) are real GEMMs of the parts
  (Re = ArBr - AiBi, Im = ArBi + AiBr), four calls of the real code path;
* exact Gaussian-integer arithmetic by brute force (Python ints);
* closed forms: alpha = i turns the product by a quarter turn exactly,
  beta = 0 never reads C (NaN in C stays out), alpha = 0 gives beta*C0.

``test_planted_mistakes_are_caught`` builds the oracle with a planted mistake
(conjugated A, alpha's imaginary part dropped, beta's imaginary sign flipped)
and checks that some pin fails.
"""
import numpy as np
import pytest

import oracle
from paper_2208_09822_gb300 import workloads as W


def _views(b, t):
    """Dense complex128 op(A), op(B), C0 of instance t."""
    M, N, K = int(b.M[t]), int(b.N[t]), int(b.K[t])

    def mat(pool, off, rows, cols, ld):
        if rows == 0 or cols == 0:
            return np.zeros((rows, cols), np.complex128)
        idx = off + np.arange(cols)[None, :] * ld + np.arange(rows)[:, None]
        return pool[idx].astype(np.complex128)

    A = mat(b.A, b.offA[t], K if b.transA[t] else M, M if b.transA[t] else K, int(b.lda[t]))
    B = mat(b.B, b.offB[t], N if b.transB[t] else K, K if b.transB[t] else N, int(b.ldb[t]))
    C = mat(b.C, b.offC[t], M, N, int(b.ldc[t]))
    return (A.T if b.transA[t] else A), (B.T if b.transB[t] else B), C


def _result(out, off, b, t):
    M, N = int(b.M[t]), int(b.N[t])
    return out[off[t]:off[t] + M * N].reshape(N, M).T


def _real_part_batch(b, which_a, which_b):
    """A real FP64 batch whose instance t is (part of A_t) x (part of B_t)
    with alpha = 1, beta = 0, in the same storage layout."""
    partA = np.real(b.A) if which_a == "re" else np.imag(b.A)
    partB = np.real(b.B) if which_b == "re" else np.imag(b.B)
    return W.Batch(np.float64, b.M, b.N, b.K, b.transA, b.transB, b.lda, b.ldb, b.ldc,
                   np.ones(b.count), np.zeros(b.count), b.offA, b.offB, b.offC,
                   np.ascontiguousarray(partA, np.float64), np.ascontiguousarray(partB, np.float64),
                   np.zeros(len(b.C), np.float64))


def pin_failures(mutant=0):
    fails = []

    # 1. numpy complex128 matmul, both component types, every case
    for dtype in (np.complex64, np.complex128):
        b = W.random_small(240, seed=21, dtype=dtype, max_dim=9, pad_max=3, misalign_max=2)
        out, off = oracle.cgemm_batch(b, mutant=mutant)
        for t in range(b.count):
            opA, opB, C0 = _views(b, t)
            ref = b.alpha[t] * (opA @ opB) + (b.beta[t] * C0 if b.beta[t] != 0 else 0)
            scale = abs(b.alpha[t]) * np.abs(opA) @ np.abs(opB) + abs(b.beta[t]) * np.abs(C0)
            if not np.all(np.abs(_result(out, off, b, t) - ref) <= 1e-14 * scale):
                fails.append(f"numpy-{np.dtype(dtype).name}")
                break

    # 2. the real oracle on the parts: Re(AB) = ArBr - AiBi, Im(AB) = ArBi + AiBr
    b = W.random_small(200, seed=22, dtype=np.complex128, max_dim=11, pad_max=2,
                       alpha=np.ones(200), beta=np.zeros(200))
    out, off = oracle.cgemm_batch(b, mutant=mutant)
    parts = {}
    for pa in ("re", "im"):
        for pb in ("re", "im"):
            parts[pa + pb], roff = oracle.gemm_batch(_real_part_batch(b, pa, pb))
    re = parts["rere"] - parts["imim"]
    im = parts["reim"] + parts["imre"]
    if not (np.array_equal(roff, off) and np.allclose(out.real, re, rtol=1e-13, atol=1e-13)
            and np.allclose(out.imag, im, rtol=1e-13, atol=1e-13)):
        fails.append("real-parts")

    # 3. Gaussian integers by brute force: exact in every format
    rng = np.random.default_rng(23)
    Ms, Ns, Ks, tas, tbs, als, bes, pads = [], [], [], [], [], [], [], []
    choices = [0, 1, -1, 1j, 1 + 1j, 2 - 1j]
    for ta in (0, 1):
        for tb in (0, 1):
            for M in range(4):
                for N in range(4):
                    for K in range(4):
                        Ms.append(M); Ns.append(N); Ks.append(K); tas.append(ta); tbs.append(tb)
                        als.append(choices[rng.integers(len(choices))])
                        bes.append(choices[rng.integers(len(choices))])
                        pads.append(rng.choice([0, 1, 3], 3))
    b = W.make_batch(Ms, Ns, Ks, tas, tbs, np.array(als, complex), np.array(bes, complex),
                     np.complex64, rng, pad=np.array(pads), dist="int")
    out, off = oracle.cgemm_batch(b, mutant=mutant)
    for t in range(b.count):
        opA, opB, C0 = _views(b, t)
        M, N, K = int(b.M[t]), int(b.N[t]), int(b.K[t])
        al, be = complex(b.alpha[t]), complex(b.beta[t])
        ok = True
        got = _result(out, off, b, t)
        for i in range(M):
            for j in range(N):
                sr = si = 0
                for k in range(K):
                    xr, xi = int(opA[i, k].real), int(opA[i, k].imag)
                    yr, yi = int(opB[k, j].real), int(opB[k, j].imag)
                    sr += xr * yr - xi * yi
                    si += xr * yi + xi * yr
                ar, ai, br, bi = int(al.real), int(al.imag), int(be.real), int(be.imag)
                er = ar * sr - ai * si
                ei = ar * si + ai * sr
                if be != 0:
                    cr, ci = int(C0[i, j].real), int(C0[i, j].imag)
                    er += br * cr - bi * ci
                    ei += br * ci + bi * cr
                if got[i, j] != complex(er, ei):
                    ok = False
        if not ok:
            fails.append("gaussian-integers")
            break

    # 4. alpha = i is a quarter turn of alpha = 1, exactly
    b1 = W.random_small(100, seed=24, dtype=np.complex128, max_dim=8, alpha=np.ones(100), beta=np.zeros(100))
    bi_ = W.random_small(100, seed=24, dtype=np.complex128, max_dim=8, alpha=np.full(100, 1j), beta=np.zeros(100))
    o1, _ = oracle.cgemm_batch(b1, mutant=mutant)
    oi, _ = oracle.cgemm_batch(bi_, mutant=mutant)
    if not np.array_equal(oi, 1j * o1):
        fails.append("alpha-i")

    # 5. beta = 0 ignores NaN in C; alpha = 0 gives beta*C0 exactly
    b = W.random_small(80, seed=25, dtype=np.complex64, max_dim=7, beta=np.zeros(80))
    b.C[:] = complex(np.nan, np.nan)
    out, _ = oracle.cgemm_batch(b, mutant=mutant)
    if np.isnan(out).any():
        fails.append("beta0-nan")
    b = W.random_small(80, seed=26, dtype=np.complex64, max_dim=7, alpha=np.zeros(80))
    out, off = oracle.cgemm_batch(b, mutant=mutant)
    for t in range(b.count):
        _, _, C0 = _views(b, t)
        if not np.array_equal(_result(out, off, b, t), b.beta[t] * C0):
            fails.append("alpha0")
            break
    return fails


def test_complex_oracle_pins_hold():
    assert pin_failures() == []


@pytest.mark.parametrize("mutant", [5, 6, 7])
def test_planted_mistakes_are_caught(mutant):
    assert pin_failures(mutant), f"planted mistake {mutant} passed every pin"


def test_complex_oracle_rejects_real_pools():
    b = W.random_small(4, seed=1)
    with pytest.raises(TypeError):
        oracle.cgemm_batch(b)
