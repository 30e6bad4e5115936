"""The library's run-time tiler (host only): exact covers, and the memops
objective of Sec. V-A checked against the oracle's Algorithm 2 and its
exhaustive search."""
import itertools
import os

import numpy as np
import pytest

from oracle import tiler_oracle as T
from paper_2208_09822_gb300 import build as B
from paper_2208_09822_gb300 import iaat


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def table1(golden_dir, typ, case):
    shapes = {}
    for line in open(os.path.join(golden_dir, "table1_kernel_shapes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t, c, h, w = line.split()
        if t == typ and c == case:
            shapes[int(h)] = int(w)
    return shapes


def covers(blocks, M, N):
    seen = np.zeros((M, N), np.int32)
    for r, c, m, n in blocks:
        assert m >= 1 and n >= 1 and r + m <= M and c + n <= N
        seen[r:r + m, c:c + n] += 1
    return bool(np.all(seen == 1))


@pytest.mark.parametrize("dtype", [iaat.IAAT_F32, iaat.IAAT_F64])
def test_gpu_tiling_is_an_exact_cover(dtype):
    for M in range(1, 81, 3):
        for N in range(1, 81, 2):
            for K in (1, 17, 80):
                assert covers(iaat.iaat_tile(dtype, 0, 0, M, N, K), M, N), (M, N, K)


def test_gpu_tiling_blocks_fit_a_variant():
    # every block of the tilers is at most 32 x 32
    for dt in (iaat.IAAT_F32, iaat.IAAT_F64):
        for M, N in itertools.product(range(1, 81, 7), range(1, 81, 5)):
            for r, c, m, n in iaat.iaat_tile(dt, 0, 0, M, N, 16):
                assert m <= 32 and n <= 32


def test_exact_tiler_worked_example(golden_dir):
    shapes = table1(golden_dir, "SGEMM", "NN")
    rows = [l.split() for l in open(os.path.join(golden_dir, "worked_example_15x15.txt"))
            if l.strip() and not l.startswith("#")]
    M, N, s_iaat = int(rows[0][0]), int(rows[0][1]), int(rows[0][2])
    blocks, s = iaat.iaat_tile_exact(M, N, list(shapes), [shapes[h] for h in shapes])
    assert s == s_iaat
    assert covers(blocks, M, N)


@pytest.mark.parametrize("typ,case", [("SGEMM", "NN"), ("SGEMM", "NT"), ("SGEMM", "TN"),
                                      ("DGEMM", "NN"), ("DGEMM", "TN")])
def test_exact_tiler_matches_exhaustive_optimum(golden_dir, typ, case):
    shapes = table1(golden_dir, typ, case)
    for M in range(1, 11):
        for N in range(1, 11):
            blocks, s = iaat.iaat_tile_exact(M, N, list(shapes), [shapes[h] for h in shapes])
            assert covers(blocks, M, N)
            for r, c, m, n in blocks:
                assert m in shapes and n <= shapes[m]
            assert s == sum(m + n for *_, m, n in blocks)
            assert s == T.min_strip_memops(M, N, shapes), (M, N)


def test_exact_tiler_never_worse_than_algorithm2(golden_dir):
    shapes = table1(golden_dir, "SGEMM", "NN")
    hs = list(shapes)
    ws = [shapes[h] for h in hs]
    for M in range(1, 81):
        for N in range(1, 81):
            _, s = iaat.iaat_tile_exact(M, N, hs, ws)
            alg2 = sum(m + n for *_, m, n in T.sgemm_nn_tile(M, N, shapes))
            assert s <= alg2, (M, N)
