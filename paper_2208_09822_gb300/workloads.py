"""Seeded synthetic small-GEMM batches.

This module draws sizes, transposition cases, leading dimensions, scalars and
matrix entries; it holds none of the GEMM arithmetic.  The library, its tests,
the oracle's tests and the benchmark all take their inputs from here.

A batch is stored as three flat pools (A, B, C) of one floating type: real
(float32 / float64) or complex (complex64 / complex128, the CGEMM and ZGEMM
types of Table I, an element being a (real, imaginary) pair).  Each
matrix of instance t starts at an element offset (offA/offB/offC) and is
stored column-major with its own leading dimension; the stored A is MxK
(transA == 0) or KxM (transA == 1), the stored B is KxN or NxK, C is MxN.
This is the layout of Sec. I and of the note under Table I (first letter of
"NN/NT/TN/TT" is A, column-major storage).

Elements outside the rows of a column (the ld padding) hold sentinels: NaN in
A and B, so any read of them poisons a result, and C_SENTINEL in C, so any
write to them can be seen.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C_SENTINEL = -7777.25

#: M, N, K values of the same-shape sweep (each of M, N and K drawn from it).
SWEEP_SIZES = (1, 2, 3, 4, 5, 7, 8, 12, 16, 24, 32, 48, 64, 80)

#: transposition cases as (transA, transB); names follow Table I.
TRANS_CASES = {"NN": (0, 0), "NT": (0, 1), "TN": (1, 0), "TT": (1, 1)}

#: Small-GEMM domain of Sec. I / Sec. VI in integer form:
#: cbrt(MNK) <= 80  <=>  MNK <= 512000, and <= 32**3 when the case is TN.
DOMAIN_MNK = 80 ** 3
DOMAIN_MNK_TN = 32 ** 3


def in_domain(M, N, K, ta, tb):
    lim = np.where((np.asarray(ta) == 1) & (np.asarray(tb) == 0),
                   DOMAIN_MNK_TN, DOMAIN_MNK)
    return np.asarray(M, np.int64) * N * K <= lim


@dataclass
class Batch:
    dtype: type
    M: np.ndarray
    N: np.ndarray
    K: np.ndarray
    transA: np.ndarray
    transB: np.ndarray
    lda: np.ndarray
    ldb: np.ndarray
    ldc: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    offA: np.ndarray
    offB: np.ndarray
    offC: np.ndarray
    A: np.ndarray
    B: np.ndarray
    C: np.ndarray
    recipe: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def count(self):
        return int(len(self.M))

    @property
    def esize(self):
        return int(np.dtype(self.dtype).itemsize)

    def storage(self, which):
        """(rows, cols, ld, off) of the stored matrices 'A', 'B' or 'C'."""
        M, N, K = self.M.astype(np.int64), self.N.astype(np.int64), self.K.astype(np.int64)
        if which == "A":
            ta = self.transA.astype(bool)
            return np.where(ta, K, M), np.where(ta, M, K), self.lda.astype(np.int64), self.offA
        if which == "B":
            tb = self.transB.astype(bool)
            return np.where(tb, N, K), np.where(tb, K, N), self.ldb.astype(np.int64), self.offB
        return M, N, self.ldc.astype(np.int64), self.offC

    @property
    def is_complex(self):
        return bool(np.issubdtype(np.dtype(self.dtype), np.complexfloating))

    def flops(self):
        """Eq. 1 numerator, sum of 2*M*N*K; complex types Eq. 2, 8*M*N*K."""
        return int((8 if self.is_complex else 2) * np.sum(self.M.astype(np.int64) * self.N * self.K))

    def algorithmic_bytes(self):
        """Bytes a GEMM must move: A, B, C written, and C read when beta != 0
        (ld padding excluded)."""
        M, N, K = self.M.astype(np.int64), self.N.astype(np.int64), self.K.astype(np.int64)
        active = (M > 0) & (N > 0)
        kread = np.where(self.alpha != 0, K, 0)
        elems = M * kread + kread * N + M * N + np.where(self.beta != 0, M * N, 0)
        return int(np.sum(np.where(active, elems, 0)) * self.esize)

    def select(self, idx):
        """A sub-batch sharing the same pools."""
        idx = np.asarray(idx)
        kw = {k: getattr(self, k)[idx] for k in (
            "M", "N", "K", "transA", "transB", "lda", "ldb", "ldc", "alpha",
            "beta", "offA", "offB", "offC")}
        return Batch(self.dtype, A=self.A, B=self.B, C=self.C,
                     recipe=self.recipe + " [subset]", **kw)


def log_uniform_int(rng, lo, hi, size):
    """floor(exp(U[ln lo, ln(hi+1)))) clipped to hi."""
    x = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size)))
    return np.minimum(x.astype(np.int64), hi)


def _layout(rows, cols, ld, align, misalign=None):
    """Element offsets for matrices packed one after another, each start
    rounded up to ``align`` elements and then moved by ``misalign``."""
    size = np.where((rows > 0) & (cols > 0), ld * cols, 0).astype(np.int64)
    off = np.zeros(len(size), dtype=np.int64)
    pos = 0
    mis = np.zeros(len(size), np.int64) if misalign is None else np.asarray(misalign, np.int64)
    # vectorised running sum of aligned slots
    slot = ((size + mis + align - 1) // align) * align
    slot = np.maximum(slot, align)
    starts = np.zeros(len(size), dtype=np.int64)
    if len(size) > 1:
        starts[1:] = np.cumsum(slot)[:-1]
    off = starts + mis
    pos = int(starts[-1] + slot[-1]) if len(size) else 0
    return off, pos + align


def _fill(pool, off, rows, cols, ld, draw, chunk=8192):
    """Write drawn values into the rows x cols part of every matrix."""
    n = len(off)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        r = rows[s:e]
        c = cols[s:e]
        cnt = r * c
        tot = int(cnt.sum())
        if tot == 0:
            continue
        inst = np.repeat(np.arange(e - s), cnt)
        first = np.zeros(e - s, np.int64)
        first[1:] = np.cumsum(cnt)[:-1]
        loc = np.arange(tot, dtype=np.int64) - first[inst]
        rr = r[inst]
        idx = off[s:e][inst] + (loc // rr) * ld[s:e][inst] + loc % rr
        pool[idx] = draw(tot, inst + s)


def make_batch(M, N, K, ta, tb, alpha, beta, dtype, rng, *, pad=None,
               dist="uniform", scale=None, align_bytes=16, misalign=None,
               recipe=""):
    """Lay out and fill a batch.

    pad: None for tight leading dimensions, else an array (n, 3) of extra
    rows for lda, ldb, ldc.  dist: 'uniform' (U[-1,1]) or 'normal' (N(0,1)).
    scale: optional per-instance factor applied to every entry of A, B, C.
    misalign: optional (n, 3) element shifts of each matrix start.
    """
    M = np.asarray(M, np.int64); N = np.asarray(N, np.int64); K = np.asarray(K, np.int64)
    n = len(M)
    ta = np.asarray(ta, np.uint8); tb = np.asarray(tb, np.uint8)
    rA = np.where(ta == 1, K, M); cA = np.where(ta == 1, M, K)
    rB = np.where(tb == 1, N, K); cB = np.where(tb == 1, K, N)
    rC, cC = M, N
    if pad is None:
        pad = np.zeros((n, 3), np.int64)
    pad = np.asarray(pad, np.int64)
    lda = np.maximum(1, rA + pad[:, 0]); ldb = np.maximum(1, rB + pad[:, 1])
    ldc = np.maximum(1, rC + pad[:, 2])
    esz = np.dtype(dtype).itemsize
    cplx = bool(np.issubdtype(np.dtype(dtype), np.complexfloating))
    align = max(1, align_bytes // esz)
    mis = [None] * 3 if misalign is None else [np.asarray(misalign)[:, i] for i in range(3)]
    offA, lenA = _layout(rA, cA, lda, align, mis[0])
    offB, lenB = _layout(rB, cB, ldb, align, mis[1])
    offC, lenC = _layout(rC, cC, ldc, align, mis[2])
    sent_ab = complex(np.nan, np.nan) if cplx else np.nan
    sent_c = complex(C_SENTINEL, C_SENTINEL) if cplx else C_SENTINEL
    A = np.full(lenA, sent_ab, dtype=dtype)
    B = np.full(lenB, sent_ab, dtype=dtype)
    C = np.full(lenC, sent_c, dtype=dtype)
    fac = None if scale is None else np.asarray(scale, np.float64)

    def draw_real(tot):
        if dist == "uniform":
            return rng.uniform(-1.0, 1.0, tot)
        if dist == "normal":
            return rng.standard_normal(tot)
        if dist == "int":
            return rng.integers(-4, 5, tot).astype(np.float64)
        raise ValueError(dist)

    def draw(tot, inst):
        # complex entries: the real parts of a chunk, then its imaginary parts
        v = draw_real(tot)
        if cplx:
            v = v + 1j * draw_real(tot)
        if fac is not None:
            v = v * fac[inst]
        return v.astype(dtype)

    _fill(A, offA, rA, cA, lda, draw)
    _fill(B, offB, rB, cB, ldb, draw)
    _fill(C, offC, rC, cC, ldc, draw)
    st = np.complex128 if cplx else np.float64
    al = np.asarray(alpha, st) * np.ones(n, st)
    be = np.asarray(beta, st) * np.ones(n, st)
    al = al.astype(dtype).astype(st)
    be = be.astype(dtype).astype(st)
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    return Batch(dtype, i32(M), i32(N), i32(K), ta, tb, i32(lda), i32(ldb),
                 i32(ldc), al, be, offA, offB, offC, A, B, C, recipe=recipe)


# --------------------------------------------------------------- workloads

def uniform16(count=10_000, seed=0):
    """10,000 FP32 NN instances of 16x16x16, ld = 16, alpha = 1, beta = 0.5,
    entries U[-1,1], seed 0."""
    rng = np.random.default_rng(seed)
    n = count
    return make_batch(np.full(n, 16), np.full(n, 16), np.full(n, 16),
                      np.zeros(n), np.zeros(n), 1.0, 0.5, np.float32, rng,
                      recipe=f"uniform16: {n} x 16^3 FP32 NN, ld=16, a=1, b=0.5, U[-1,1], seed {seed}")


def sweep_shapes(case):
    """(M, N, K) triples of the same-shape sweep that lie in the domain."""
    ta, tb = TRANS_CASES[case]
    out = []
    for M in SWEEP_SIZES:
        for N in SWEEP_SIZES:
            for K in SWEEP_SIZES:
                if in_domain(M, N, K, ta, tb):
                    out.append((M, N, K))
    return out


def sweep(case, shape, dtype=np.float32, count=4096, seed=1, decades=None):
    """``count`` same-shape instances, tight ld, alpha = 1.25, beta = -0.75,
    entries U[-1,1] (seed 1).  ``decades`` = 3 scales every entry of an
    instance by 10**U[-3,3] (the precision study)."""
    ta, tb = TRANS_CASES[case]
    M, N, K = shape
    rng = np.random.default_rng(seed)
    n = count
    scale = None
    if decades:
        scale = 10.0 ** rng.uniform(-decades, decades, n)
    return make_batch(np.full(n, M), np.full(n, N), np.full(n, K),
                      np.full(n, ta), np.full(n, tb), 1.25, -0.75, dtype, rng,
                      scale=scale,
                      recipe=f"sweep {case} {M}x{N}x{K} x{n} {np.dtype(dtype).name} seed {seed}"
                             + (f" scale 10^U[-{decades},{decades}]" if decades else ""))


def sweep_mixed(case, dtype=np.float32, per_shape=2, seed=1, decades=None):
    """Every in-domain sweep shape of one case, ``per_shape`` instances each,
    in one batch (the parity-test form of the sweep)."""
    ta, tb = TRANS_CASES[case]
    shapes = sweep_shapes(case)
    rng = np.random.default_rng(seed)
    arr = np.repeat(np.asarray(shapes, np.int64), per_shape, axis=0)
    n = len(arr)
    scale = 10.0 ** rng.uniform(-decades, decades, n) if decades else None
    return make_batch(arr[:, 0], arr[:, 1], arr[:, 2], np.full(n, ta),
                      np.full(n, tb), 1.25, -0.75, dtype, rng, scale=scale,
                      recipe=f"sweep-mixed {case} {np.dtype(dtype).name} x{per_shape}/shape seed {seed}")


def uneven(count=200_000, seed=2, dtype=np.float32):
    """The uneven grouped batch: M, N, K log-uniform integers on [1, 80]
    (TN instances redrawn until MNK <= 32768), case uniform over
    NN/NT/TN/TT, ld = rows + U{0..7}, alpha, beta ~ U[-2,2] rounded to the
    type, entries N(0,1), seed 2."""
    rng = np.random.default_rng(seed)
    n = count
    M = log_uniform_int(rng, 1, 80, n)
    N = log_uniform_int(rng, 1, 80, n)
    K = log_uniform_int(rng, 1, 80, n)
    case = rng.integers(0, 4, n)
    ta = (case >> 1) & 1
    tb = case & 1
    while True:
        bad = np.nonzero(~in_domain(M, N, K, ta, tb))[0]
        if len(bad) == 0:
            break
        M[bad] = log_uniform_int(rng, 1, 80, len(bad))
        N[bad] = log_uniform_int(rng, 1, 80, len(bad))
        K[bad] = log_uniform_int(rng, 1, 80, len(bad))
    pad = rng.integers(0, 8, (n, 3))
    alpha = rng.uniform(-2, 2, n)
    beta = rng.uniform(-2, 2, n)
    return make_batch(M, N, K, ta, tb, alpha, beta, dtype, rng, pad=pad,
                      dist="normal",
                      recipe=f"uneven: {n} instances, M,N,K log-U[1,80], cases uniform, "
                             f"ld=rows+U{{0..7}}, a,b~U[-2,2], N(0,1), seed {seed}")


def fc64(count=100_000, seed=4):
    """FP64 batch shaped like fully connected layers: M in {32, 64}, K and N
    log-uniform on [8, 80], NN or TN 50/50 (TN redrawn until MNK <= 32768),
    alpha = 1, beta in {0, 1} 50/50, entries U[-1,1], seed 4."""
    rng = np.random.default_rng(seed)
    n = count
    M = rng.choice(np.array([32, 64]), n)
    K = log_uniform_int(rng, 8, 80, n)
    N = log_uniform_int(rng, 8, 80, n)
    ta = rng.integers(0, 2, n)
    tb = np.zeros(n, np.int64)
    while True:
        bad = np.nonzero(~in_domain(M, N, K, ta, tb))[0]
        if len(bad) == 0:
            break
        M[bad] = rng.choice(np.array([32, 64]), len(bad))
        K[bad] = log_uniform_int(rng, 8, 80, len(bad))
        N[bad] = log_uniform_int(rng, 8, 80, len(bad))
    beta = rng.integers(0, 2, n).astype(np.float64)
    return make_batch(M, N, K, ta, tb, 1.0, beta, np.float64, rng,
                      recipe=f"fc64: {n} FP64, M in {{32,64}}, K,N log-U[8,80], NN/TN, "
                             f"a=1, b in {{0,1}}, U[-1,1], seed {seed}")


def uneven_complex(count=100_000, seed=5, dtype=np.complex64):
    """The uneven batch in a complex type (CGEMM: complex64, ZGEMM:
    complex128): M, N, K log-uniform integers on [1, 80] (TN redrawn until
    MNK <= 32768), case uniform, ld = rows + U{0..7}, alpha and beta with
    both parts ~ U[-2,2], entries with both parts N(0,1), seed 5."""
    rng = np.random.default_rng(seed)
    n = count
    M = log_uniform_int(rng, 1, 80, n)
    N = log_uniform_int(rng, 1, 80, n)
    K = log_uniform_int(rng, 1, 80, n)
    case = rng.integers(0, 4, n)
    ta = (case >> 1) & 1
    tb = case & 1
    while True:
        bad = np.nonzero(~in_domain(M, N, K, ta, tb))[0]
        if len(bad) == 0:
            break
        M[bad] = log_uniform_int(rng, 1, 80, len(bad))
        N[bad] = log_uniform_int(rng, 1, 80, len(bad))
        K[bad] = log_uniform_int(rng, 1, 80, len(bad))
    pad = rng.integers(0, 8, (n, 3))
    alpha = rng.uniform(-2, 2, n) + 1j * rng.uniform(-2, 2, n)
    beta = rng.uniform(-2, 2, n) + 1j * rng.uniform(-2, 2, n)
    return make_batch(M, N, K, ta, tb, alpha, beta, dtype, rng, pad=pad,
                      dist="normal",
                      recipe=f"uneven-complex: {n} {np.dtype(dtype).name} instances, M,N,K log-U[1,80], "
                             f"cases uniform, ld=rows+U{{0..7}}, a,b parts ~U[-2,2], N(0,1) parts, seed {seed}")


def random_small(count, seed, dtype=np.float32, max_dim=12, pad_max=3,
                 dist="uniform", misalign_max=0, alpha=None, beta=None):
    """Small random instances of every case (tests): dims U{0..max_dim},
    random ld padding and optional start misalignment.  Complex types draw
    complex alpha and beta (both parts U[-2,2])."""
    rng = np.random.default_rng(seed)
    n = count
    M = rng.integers(0, max_dim + 1, n)
    N = rng.integers(0, max_dim + 1, n)
    K = rng.integers(0, max_dim + 1, n)
    case = rng.integers(0, 4, n)
    ta = (case >> 1) & 1
    tb = case & 1
    pad = rng.integers(0, pad_max + 1, (n, 3))
    mis = rng.integers(0, misalign_max + 1, (n, 3)) if misalign_max else None
    cplx = np.issubdtype(np.dtype(dtype), np.complexfloating)
    if alpha is None:
        al = rng.uniform(-2, 2, n)
        al = al + 1j * rng.uniform(-2, 2, n) if cplx else al
    else:
        al = alpha
    if beta is None:
        be = rng.uniform(-2, 2, n)
        be = be + 1j * rng.uniform(-2, 2, n) if cplx else be
    else:
        be = beta
    return make_batch(M, N, K, ta, tb, al, be, dtype, rng, pad=pad, dist=dist,
                      misalign=mis, recipe=f"random_small seed {seed}")
