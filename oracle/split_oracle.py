"""Emulation oracle of the tensor-core paths -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; it imports nothing from the library.

The tensor-core paths do not compute the plain GEMM: they first round the
FP32 operands to narrower formats and add a fixed set of products.  This
module takes those steps in order, in numpy, with the sums in FP64 (the
paths accumulate in FP32, so they differ from it only by FP32 accumulation
error):

* 3xBF16:  X = Xh + Xl, Xh = bf16(X), Xl = bf16(X - Xh);  Ah Bh + Ah Bl + Al Bh
* 6xBF16:  X = Xh + Xm + Xl, each term the BF16 rounding of what the terms
           before it leave;  the six products of order up to two
           (mm, lh, hl, mh, hm, hh)
* TF32:    tf32(A) tf32(B), tf32 = round to 10 explicit mantissa bits
* FP16:    fp16(A) fp16(B)

bf16 and tf32 round to nearest, ties to even, on the FP32 bit pattern (Inf
and NaN pass unchanged); fp16 is numpy's IEEE half conversion (subnormals
included).  The differences X - Xh are exact in FP32.  Then
C = alpha * sum + beta * C0 in FP64, with the GEMM conventions of the plain
oracle (beta == 0 never reads C0, alpha == 0 or K == 0 skips the sum).
"""
from __future__ import annotations

import numpy as np

PRECISIONS = ("3xbf16", "6xbf16", "tf32", "fp16")


def _round_bits(x, drop):
    """Round FP32 values to nearest, ties to even, keeping all but the low
    `drop` bits of the significand (Inf / NaN unchanged)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    special = (u & 0x7F800000) == 0x7F800000
    half = np.uint64((1 << (drop - 1)) - 1)
    mask = np.uint64((0xFFFFFFFF >> drop) << drop)
    r = (u + half + ((u >> np.uint64(drop)) & np.uint64(1))) & mask
    r = np.where(special, u, r).astype(np.uint32)
    return r.view(np.float32)


def bf16_rn(x):
    """FP32 -> BF16 (8 significant bits), nearest-even, as FP32 values."""
    return _round_bits(x, 16)


def tf32_rn(x):
    """FP32 -> TF32 (11 significant bits), nearest-even, as FP32 values."""
    return _round_bits(x, 13)


def fp16_rn(x):
    """FP32 -> IEEE half, nearest-even, as FP32 values."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def split_terms(x, precision):
    """The operand terms of one path (float32 arrays, summing to about x)."""
    x = np.asarray(x, dtype=np.float32)
    if precision == "3xbf16":
        h = bf16_rn(x)
        return [h, bf16_rn(x - h)]
    if precision == "6xbf16":
        h = bf16_rn(x)
        r = x - h
        m = bf16_rn(r)
        return [h, m, bf16_rn(r - m)]
    if precision == "tf32":
        return [tf32_rn(x)]
    if precision == "fp16":
        return [fp16_rn(x)]
    raise ValueError(precision)


#: (term of op(A), term of op(B)) of every product a path adds
PRODUCTS = {
    "3xbf16": ((0, 0), (0, 1), (1, 0)),
    "6xbf16": ((0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)),
    "tf32": ((0, 0),),
    "fp16": ((0, 0),),
}


def _dense(pool, off, rows, cols, ld):
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols), np.float32)
    idx = off + np.arange(cols)[None, :] * ld + np.arange(rows)[:, None]
    return pool[idx]


def tc_gemm_batch(batch, precision, idx=None, products=None):
    """What the tensor-core path `precision` computes for instances `idx` of
    an FP32 ``workloads.Batch``, in FP64.  Returns (out, off) like
    ``oracle.gemm_batch``.  `products` overrides the product list (pin
    tests plant mistakes through it)."""
    prods = PRODUCTS[precision] if products is None else products
    if idx is None:
        idx = np.arange(batch.count)
    idx = np.asarray(idx, dtype=np.int64)
    sizes = batch.M[idx].astype(np.int64) * batch.N[idx].astype(np.int64)
    off = np.zeros(len(idx), np.int64)
    if len(idx) > 1:
        off[1:] = np.cumsum(sizes)[:-1]
    out = np.zeros(int(sizes.sum()) if len(idx) else 0, np.float64)
    for j, t in enumerate(idx):
        M, N, K = int(batch.M[t]), int(batch.N[t]), int(batch.K[t])
        if M == 0 or N == 0:
            continue
        ta, tb = int(batch.transA[t]), int(batch.transB[t])
        alpha, beta = float(batch.alpha[t]), float(batch.beta[t])
        acc = np.zeros((M, N), np.float64)
        if alpha != 0.0 and K > 0:
            A = _dense(batch.A, batch.offA[t], K if ta else M, M if ta else K, int(batch.lda[t]))
            B = _dense(batch.B, batch.offB[t], N if tb else K, K if tb else N, int(batch.ldb[t]))
            opA = A.T if ta else A
            opB = B.T if tb else B
            ta_terms = [a.astype(np.float64) for a in split_terms(opA, precision)]
            tb_terms = [b.astype(np.float64) for b in split_terms(opB, precision)]
            for ia, ib in prods:
                acc += ta_terms[ia] @ tb_terms[ib]
        res = alpha * acc
        if beta != 0.0:
            res = res + beta * _dense(batch.C, batch.offC[t], M, N, int(batch.ldc[t])).astype(np.float64)
        out[off[j]:off[j] + M * N] = res.T.ravel()
    return out, off
