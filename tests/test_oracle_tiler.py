"""Pins for the tiling oracle (Algorithm 2, Sec. V-A), CPU only."""
import os

import pytest

from oracle import tiler_oracle as T


def load_shapes(golden_dir, typ, case):
    shapes = {}
    with open(os.path.join(golden_dir, "table1_kernel_shapes.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t, c, h, w = line.split()
            if t == typ and c == case:
                shapes[int(h)] = int(w)
    return shapes


@pytest.fixture(scope="module")
def nn_shapes(golden_dir):
    return load_shapes(golden_dir, "SGEMM", "NN")


def _covers_exactly(blocks, M, N, shapes):
    seen = [[0] * N for _ in range(M)]
    for r, c, m, n in blocks:
        if m not in shapes or not (1 <= n <= shapes[m]):
            return False
        for i in range(r, r + m):
            for j in range(c, c + n):
                if i >= M or j >= N:
                    return False
                seen[i][j] += 1
    return all(v == 1 for row in seen for v in row)


def test_worked_example_15x15(golden_dir, nn_shapes):
    with open(os.path.join(golden_dir, "worked_example_15x15.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    M, N, s_iaat, const, _s_trad = map(int, rows[0])
    blocks = T.sgemm_nn_tile(M, N, nn_shapes)
    assert _covers_exactly(blocks, M, N, nn_shapes)
    assert sum(m + n for _, _, m, n in blocks) == s_iaat
    for K in (1, 7, 80):
        assert T.memops(blocks, M, N, K) == s_iaat * K + const
    # the paper's tiling is also the best row-strip tiling for this size
    assert T.min_strip_memops(M, N, nn_shapes) == s_iaat


def test_exact_cover_every_size(nn_shapes):
    for M in range(1, 81):
        for N in range(1, 81):
            blocks = T.sgemm_nn_tile(M, N, nn_shapes)
            assert _covers_exactly(blocks, M, N, nn_shapes), (M, N)


def test_printed_special_cases(nn_shapes):
    def strips(blocks):
        return sorted({(r, m) for r, _, m, _ in blocks})
    # M == 9, N > 13: strips 4, 3, 2
    assert [m for _, m in strips(T.sgemm_nn_tile(9, 20, nn_shapes))] == [4, 3, 2]
    # M in {10, 11}: 8 then M - 8; the 8-row strip uses widths <= 8
    for M in (10, 11):
        b = T.sgemm_nn_tile(M, 30, nn_shapes)
        assert [m for _, m in strips(b)] == [8, M - 8]
        assert max(n for _, _, m, n in b if m == 8) <= 8
    # M == 12: one 12-row strip of widths <= 6
    b = T.sgemm_nn_tile(12, 40, nn_shapes)
    assert {m for _, _, m, _ in b} == {12} and max(n for *_, n in b) <= 6
    # N <= 13: one column of width N, tallest kernel that holds it
    b = T.sgemm_nn_tile(40, 3, nn_shapes)
    assert {n for *_, n in b} == {3} and max(m for _, _, m, _ in b) == 16


def test_tile_single_dim():
    assert T.tile_single_dim(26, range(1, 14)) == [(13, 2)]
    assert T.tile_single_dim(15, range(1, 14)) == [(8, 1), (7, 1)]   # 13+2 averaged
    assert T.tile_single_dim(20, range(1, 14)) == [(13, 1), (7, 1)]  # 7 is not too small
    assert T.tile_single_dim(19, range(1, 14)) == [(10, 1), (9, 1)]  # 6 < 13/2 is
    assert T.tile_single_dim(5, [1, 2, 3, 4]) == [(3, 1), (2, 1)]
    assert T.tile_single_dim(4, [1, 2, 3, 4]) == [(4, 1)]
    for L in range(1, 60):
        runs = T.tile_single_dim(L, range(1, 14))
        assert sum(d * c for d, c in runs) == L


def test_alg2_never_beats_exhaustive_optimum(nn_shapes):
    for M in range(1, 13):
        for N in range(1, 13):
            blocks = T.sgemm_nn_tile(M, N, nn_shapes)
            assert sum(m + n for *_, m, n in blocks) >= T.min_strip_memops(M, N, nn_shapes)


def test_memops_counts_loads():
    """Count loads of a blocked GEMM one by one: each block reads its m x K
    slice of A and K x n slice of B, and C is read and written once."""
    blocks = [(0, 0, 4, 3), (0, 3, 4, 2), (4, 0, 2, 5)]
    M, N, K = 6, 5, 9
    loads = 0
    for r, c, m, n in blocks:
        for k in range(K):
            loads += m   # one column of the A block
            loads += n   # one row of the B block
    loads += 2 * M * N
    assert T.memops(blocks, M, N, K) == loads


def test_blocks_ab_compute_the_product(nn_shapes):
    """blocksA / blocksB are the slices of A and B each C block reads: a
    blocked product that takes, for every C block, the A rows and B columns
    blocks_ab names equals A @ B, and their element count is the memops
    count of the tiling minus the 2*M*N values of C."""
    import numpy as np
    rng = np.random.default_rng(0)
    for M, N, K in ((15, 15, 7), (9, 20, 3), (40, 3, 5), (29, 31, 4), (13, 14, 2)):
        A = rng.integers(-4, 5, (M, K))
        B = rng.integers(-4, 5, (K, N))
        blocks = T.sgemm_nn_tile(M, N, nn_shapes)
        ba, bb = T.blocks_ab(blocks, K)
        assert len(ba) == len(bb) == len(blocks)
        C = np.zeros((M, N), np.int64)
        for (r, c, m, n), (ra, ma, ka), (cb, nb, kb) in zip(blocks, ba, bb):
            assert (ra, ma, ka) == (r, m, K) and (cb, nb, kb) == (c, n, K)
            C[r:r + m, c:c + n] += A[ra:ra + ma, :ka] @ B[:kb, cb:cb + nb]
        assert np.array_equal(C, A @ B)
        loads = sum(m * k for _, m, k in ba) + sum(n * k for _, n, k in bb)
        assert loads + 2 * M * N == T.memops(blocks, M, N, K)


def test_remainder_of_one_row(nn_shapes):
    """M = 4q + 1 beyond 12 rows: one 4-row strip gives way to a 3- and a
    2-row strip, each cut across N with the widths its height's kernels
    reach (reading 6: 13 for both)."""
    for M in (13, 17, 41, 77):
        b = T.sgemm_nn_tile(M, 40, nn_shapes)
        hs = sorted({(r, m) for r, _, m, _ in b})
        assert [m for _, m in hs][-2:] == [3, 2], (M, hs)
        assert max(n for _, _, m, n in b if m == 3) == 13
        assert all(m != 1 for _, _, m, _ in b)
