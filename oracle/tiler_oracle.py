"""Reference for the run-time tiling stage -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this module.  It shares nothing with the library.

Contents
--------
* ``tile_single_dim``  -- the one-dimension splitter used by Algorithm 2
  (Sec. V-A, "TileSingleDim"): greedy runs of the largest size, and a last
  piece that is "too small" averaged with the one before it.
* ``sgemm_nn_tile``    -- Algorithm 2 (Sec. V-A), the SGEMM_NN tiler, taken
  case by case in the paper's order and notation.
* ``memops``           -- the "Minimal Memops" count of Sec. V-A:
  (m_0+n_0+...+m_a+n_a)*K + 2*M*N values moved between cache and registers.
* ``min_strip_memops`` -- exhaustive search over every row-strip tiling (each
  strip split into blocks) for the smallest sum(m_i+n_i), tiny sizes only.

Readings where the paper is silent or garbled (the builder's choices):
1. A remainder that is not itself a kernel height (Algorithm 2, N <= 13 branch)
   is tiled again with the same rule: the largest height whose kernel row
   holds width N, repeated while it fits.
2. TileSingleDim's "too small" is "less than half of the largest piece"; the
   last full piece and the remainder are then replaced by the two halves of
   their sum (ceil, floor).  This leaves sum(n) and the piece count unchanged.
3. ExtendTo8 merges pairs of 4-row strips into 8-row strips; ExtendTo16 merges
   groups of four into 16-row strips, and a leftover of three, two or one
   4-row strips becomes one 12-, 8- or 4-row strip.  The 15x15 example needs
   three 4-row strips to become one 12-row strip.
4. CompareLessMemops keeps the first candidate on a tie.
5. "2mn" in the memops formula is 2*M*N (one load and one store of C); the
   worked example's 450 = 2*15*15 fixes this.

Shape sets are passed in as {height: max_width}: a kernel m_c x n_c exists for
every width 1..max_width of that height (that is how every row of Table I is
written).
"""
from __future__ import annotations

from itertools import product as _product


def tile_single_dim(length, sizes):
    """TileSingleDim(len, sizes) of Sec. V-A: return runs [(dim, nums), ...].

    ``sizes`` is a contiguous range 1..s in every use the paper makes.
    """
    if length <= 0:
        return []
    usable = [s for s in sizes if s <= length]
    smax = max(usable)
    nums, rem = divmod(length, smax)
    runs = [(smax, nums)]
    if rem:
        if 2 * rem < smax:
            # the last piece is too small: average it with the one before
            total = smax + rem
            hi, lo = (total + 1) // 2, total // 2
            runs = [(smax, nums - 1)] if nums > 1 else []
            if hi == lo:
                runs.append((hi, 2))
            else:
                runs.append((hi, 1))
                runs.append((lo, 1))
        else:
            runs.append((rem, 1))
    return [(d, c) for d, c in runs if c > 0]


def _widths(maxw):
    return list(range(1, maxw + 1))


def _combine(mruns, nlists):
    """Combine(m, n): strip runs m[r] = (height, count), each strip split by
    the column runs nlists[r]; return blocks (row0, col0, m_c, n_c)."""
    blocks = []
    row = 0
    for (h, cnt), nruns in zip(mruns, nlists):
        for _ in range(cnt):
            col = 0
            for w, wc in nruns:
                for _ in range(wc):
                    blocks.append((row, col, h, w))
                    col += w
            row += h
    return blocks


def _strip_sum(blocks):
    return sum(m + n for _, _, m, n in blocks)


def _extend(q, group):
    """ExtendTo8 (group=2) / ExtendTo16 (group=4) on q strips of height 4."""
    runs = []
    full, left = divmod(q, group)
    if full:
        runs.append((4 * group, full))
    if left:
        runs.append((4 * left, 1))
    return runs


def sgemm_nn_tile(M, N, shapes):
    """Algorithm 2 (Sec. V-A): SGEMM_NN tile algorithm.

    ``shapes`` is the SGEMM_NN row of Table I as {height: max_width}.
    Returns blocksC as a list of (row0, col0, m_c, n_c); blocksA / blocksB
    follow from it (rows row0.. of A with all K columns, columns col0.. of B
    with all K rows) and are returned by ``blocks_ab``.
    """
    if M <= 0 or N <= 0:
        return []
    heights = sorted(shapes, reverse=True)
    if N <= 13:
        # m_1: largest kernel height whose row holds width N; I = floor(M/m_1)
        def tallest(limit):
            return max(h for h in heights if h <= limit and shapes[h] >= N)
        m1 = tallest(max(heights))
        I = M // m1
        mruns = [(m1, I)] if I else []
        rem = M - m1 * I
        while rem:  # reading 1: the remainder tiled with the same rule
            h = tallest(rem)
            c = rem // h
            mruns.append((h, c))
            rem -= h * c
        nlists = [[(N, 1)] for _ in mruns]
        return _combine(mruns, nlists)
    w13, w8, w6 = _widths(13), _widths(8), _widths(6)
    if M < 8:
        mruns = tile_single_dim(M, [1, 2, 3, 4])
        nlists = [tile_single_dim(N, w13)]
        if len(mruns) == 2:
            nlists.append(tile_single_dim(N, w13))
        return _combine(mruns, nlists)
    if M == 9:
        mruns = [(4, 1), (3, 1), (2, 1)]
        nlists = [tile_single_dim(N, w13) for _ in range(3)]
        return _combine(mruns, nlists)
    if M < 12:
        mruns = [(8, 1)]
        nlists = [tile_single_dim(N, w8)]
        if M - 8:
            mruns.append((M - 8, 1))
            nlists.append(tile_single_dim(N, w13))
        return _combine(mruns, nlists)
    if M == 12:
        return _combine([(12, 1)], [tile_single_dim(N, w6)])
    # M > 12
    q = M // 4
    r = M - 4 * q
    m2 = [(r, 1)] if r else []
    n2 = [tile_single_dim(N, w13)] if r else []
    if r == 1:
        q -= 1
        m2 = [(3, 1), (2, 1)]
        n2 = [tile_single_dim(N, w8), tile_single_dim(N, w13)]
    m8 = _extend(q, 2)
    m16 = _extend(q, 4)
    n8 = [tile_single_dim(N, _widths(shapes[h])) for h, _ in m8]
    n16 = [tile_single_dim(N, _widths(shapes[h])) for h, _ in m16]
    c1 = _combine(m8, n8)
    c2 = _combine(m16, n16)
    best = c2 if _strip_sum(c2) < _strip_sum(c1) else c1  # reading 4
    top = 4 * q
    tail = [(row + top, col, m, n) for row, col, m, n in _combine(m2, n2)]
    return best + tail


def blocks_ab(blocksC, K):
    """blocksA / blocksB of Algorithm 2: the A rows and B columns each C
    block reads, as (row0, m_c, K) and (col0, n_c, K)."""
    return ([(r, m, K) for r, _, m, _ in blocksC],
            [(c, n, K) for _, c, _, n in blocksC])


def memops(blocksC, M, N, K):
    """Sec. V-A "Minimal Memops": (sum_i m_i + n_i) * K + 2*M*N (reading 5)."""
    return _strip_sum(blocksC) * K + 2 * M * N


def _compositions(n, parts):
    """Every ordered split of n into summands drawn from ``parts``."""
    if n == 0:
        yield ()
        return
    for p in parts:
        if p <= n:
            for rest in _compositions(n - p, parts):
                yield (p,) + rest


def min_strip_memops(M, N, shapes):
    """Smallest sum(m_i + n_i) over every exact tiling of an MxN C into row
    strips whose heights are kernel heights, each strip split into blocks of
    widths that height's kernels support.  Exhaustive; keep M, N <= ~16."""
    best_strip = {}
    for h, maxw in shapes.items():
        widths = list(range(1, maxw + 1))
        best_strip[h] = min(len(c) * h + N for c in _compositions(N, widths))
    heights = sorted(shapes)
    return min(sum(best_strip[h] for h in c) for c in _compositions(M, heights))
