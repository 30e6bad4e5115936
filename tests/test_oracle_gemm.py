"""Pins for the FP64 GEMM oracle (CPU only).

The oracle is the GEMM definition of Sec. I (C = alpha*op(A)*op(B) + beta*C,
column-major, NN/NT/TN/TT per the note under Table I).  Each test pins it to
something other than itself: a library routine (numpy matmul), exact integer
arithmetic by brute force, closed forms (identity, permutation, rank-1) and the
transpose identity.  ``test_planted_mistakes_are_caught`` compiles the oracle
with a planted mistake and checks that the pins fail.
"""
import numpy as np
import pytest

import oracle
from paper_2208_09822_gb300 import workloads as W


def _instance_views(b, t):
    """Dense float64 op(A), op(B), C0 of instance t of a batch."""
    M, N, K = int(b.M[t]), int(b.N[t]), int(b.K[t])

    def mat(pool, off, rows, cols, ld):
        if rows == 0 or cols == 0:
            return np.zeros((rows, cols))
        idx = off + np.arange(cols)[None, :] * ld + np.arange(rows)[:, None]
        return pool[idx].astype(np.float64)

    A = mat(b.A, b.offA[t], K if b.transA[t] else M, M if b.transA[t] else K, int(b.lda[t]))
    B = mat(b.B, b.offB[t], N if b.transB[t] else K, K if b.transB[t] else N, int(b.ldb[t]))
    C = mat(b.C, b.offC[t], M, N, int(b.ldc[t]))
    opA = A.T if b.transA[t] else A
    opB = B.T if b.transB[t] else B
    return opA, opB, C


def _result(out, off, b, t, j=None):
    j = t if j is None else j
    M, N = int(b.M[t]), int(b.N[t])
    return out[off[j]:off[j] + M * N].reshape(N, M).T


def pin_failures(mutant=0):
    """Run the pins against an oracle build; return the names that fail."""
    fails = []

    # 1. library special case: numpy matmul in float64
    for dtype in (np.float32, np.float64):
        b = W.random_small(300, seed=11, dtype=dtype, max_dim=9, pad_max=3,
                           misalign_max=3)
        out, off = oracle.gemm_batch(b, mutant=mutant)
        for t in range(b.count):
            opA, opB, C0 = _instance_views(b, t)
            ref = b.alpha[t] * (opA @ opB) + (b.beta[t] * C0 if b.beta[t] != 0 else 0)
            got = _result(out, off, b, t)
            scale = abs(b.alpha[t]) * np.abs(opA) @ np.abs(opB) + abs(b.beta[t]) * np.abs(C0)
            if not np.all(np.abs(got - ref) <= 1e-14 * scale + 0.0):
                fails.append(f"numpy-{np.dtype(dtype).name}")
                break

    # 2. brute force with exact integers: every case, M,N,K in 0..4, pads
    Ms, Ns, Ks, tas, tbs, als, bes, pads = [], [], [], [], [], [], [], []
    rng = np.random.default_rng(5)
    for ta in (0, 1):
        for tb in (0, 1):
            for M in range(5):
                for N in range(5):
                    for K in range(5):
                        Ms.append(M); Ns.append(N); Ks.append(K)
                        tas.append(ta); tbs.append(tb)
                        als.append(rng.choice([0, 1, -1, 2]))
                        bes.append(rng.choice([0, 1, -1, 2]))
                        pads.append(rng.choice([0, 1, 3], 3))
    b = W.make_batch(Ms, Ns, Ks, tas, tbs, np.array(als, float),
                     np.array(bes, float), np.float32, rng, pad=np.array(pads),
                     dist="int")
    out, off = oracle.gemm_batch(b, mutant=mutant)
    for t in range(b.count):
        opA, opB, C0 = _instance_views(b, t)
        M, N, K = int(b.M[t]), int(b.N[t]), int(b.K[t])
        al, be = int(b.alpha[t]), int(b.beta[t])
        got = _result(out, off, b, t)
        ok = True
        for i in range(M):
            for j in range(N):
                s = 0
                for k in range(K):
                    s += int(opA[i, k]) * int(opB[k, j])
                exact = al * s + (be * int(C0[i, j]) if be != 0 else 0)
                if got[i, j] != exact:
                    ok = False
        if not ok:
            fails.append("brute-force-integers")
            break

    # 3. closed forms on structured operands
    n = 6
    rng = np.random.default_rng(7)
    b = W.make_batch([n] * 4, [5] * 4, [n] * 4, [0, 0, 1, 1], [0, 1, 0, 1],
                     1.5, -0.5, np.float64, rng, pad=rng.integers(0, 3, (4, 3)))
    perm = rng.permutation(n)
    P = np.eye(n)[perm]          # op(A) = P  (P @ X permutes rows of X)
    for t in range(4):
        rows = n
        idx = b.offA[t] + np.arange(n)[None, :] * b.lda[t] + np.arange(rows)[:, None]
        b.A[idx] = (P.T if b.transA[t] else P)
    out, off = oracle.gemm_batch(b, mutant=mutant)
    for t in range(4):
        _, opB, C0 = _instance_views(b, t)
        expect = 1.5 * opB[perm, :] + (-0.5) * C0
        if not np.array_equal(_result(out, off, b, t), expect):
            fails.append("permutation")
            break

    # rank-1: K = 1 gives alpha * a b^T + beta * C0 element-wise (exact in FP64)
    b = W.make_batch([7, 3], [4, 9], [1, 1], [0, 1], [1, 0], 0.75, 2.0,
                     np.float64, np.random.default_rng(8))
    out, off = oracle.gemm_batch(b, mutant=mutant)
    for t in range(2):
        opA, opB, C0 = _instance_views(b, t)
        expect = 0.75 * np.outer(opA[:, 0], opB[0, :]) + 2.0 * C0
        if not np.array_equal(_result(out, off, b, t), expect):
            fails.append("rank-1")
            break

    # alpha = 0 gives beta*C0 exactly; beta = 0 never reads C0 (NaN there)
    b = W.make_batch([5, 5], [6, 6], [4, 4], [0, 1], [1, 0], [0.0, 1.0],
                     [3.0, 0.0], np.float32, np.random.default_rng(9))
    for t in range(2):
        _, _, _ = _instance_views(b, t)
    idx = b.offC[1] + np.arange(6)[None, :] * b.ldc[1] + np.arange(5)[:, None]
    b.C[idx] = np.nan
    out, off = oracle.gemm_batch(b, mutant=mutant)
    _, _, C0 = _instance_views(b, 0)
    if not np.array_equal(_result(out, off, b, 0), 3.0 * C0):
        fails.append("alpha-zero")
    if np.isnan(_result(out, off, b, 1)).any():
        fails.append("beta-zero-nan")

    # transpose identity: (op(A) op(B))^T = op(B)^T op(A)^T.  NN(A,B) must
    # equal the transpose of TT(B,A) with M and N swapped, using the same
    # stored arrays.
    rng = np.random.default_rng(10)
    M, N, K = 5, 7, 6
    A = rng.uniform(-1, 1, (M, K)); B = rng.uniform(-1, 1, (K, N))
    Apool = np.concatenate([A.T.ravel(), B.T.ravel()])   # column-major
    offA, offB = 0, M * K
    bb = W.Batch(np.float64, M=np.array([M, N], np.int32), N=np.array([N, M], np.int32),
                 K=np.array([K, K], np.int32), transA=np.array([0, 1], np.uint8),
                 transB=np.array([0, 1], np.uint8), lda=np.array([M, K], np.int32),
                 ldb=np.array([K, M], np.int32), ldc=np.array([M, N], np.int32),
                 alpha=np.ones(2), beta=np.zeros(2), offA=np.array([offA, offB]),
                 offB=np.array([offB, offA]), offC=np.array([0, 0]), A=Apool, B=Apool,
                 C=np.zeros(M * N))
    out, off = oracle.gemm_batch(bb, mutant=mutant)
    nn = out[off[0]:off[0] + M * N].reshape(N, M).T
    tt = out[off[1]:off[1] + M * N].reshape(M, N).T
    if np.max(np.abs(nn - tt.T)) > 1e-14:
        fails.append("transpose-identity")
    return fails


def test_oracle_pins_hold():
    assert pin_failures(0) == []


@pytest.mark.parametrize("mutant", [1, 2, 3, 4])
def test_planted_mistakes_are_caught(mutant):
    assert pin_failures(mutant), f"planted mistake {mutant} passed every pin"


def test_oracle_rejects_negative_sizes():
    b = W.random_small(3, seed=1)
    b.M[1] = -1
    with pytest.raises(ValueError):
        oracle.gemm_batch(b)
