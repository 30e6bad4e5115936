"""Reference for the run-time tiling stage -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this module.  It shares nothing with the library.

Contents
--------
* ``tile_single_dim``  -- the one-dimension splitter of Sec. V-A
  ("TileSingleDim"): as many pieces of the largest usable size as fit, and a
  last piece that is "too small" averaged with the one before it.
* ``sgemm_nn_tile``    -- the SGEMM_NN tiling of C (Sec. V-A, Algorithm 2),
  written from the section's rules: narrow C (N <= 13) is one column of
  width N cut into the tallest rows that width allows; wide C is cut into
  row strips built from 4-row strips with 1-, 2- and 3-row strips for the
  remainder (merged into 8- or 16-row strips when M > 12, whichever moves
  fewer values), and every strip is cut across N into the widest blocks
  its height allows.
* ``blocks_ab``        -- the blocks of A and B the C blocks read.
* ``memops``           -- the "Minimal Memops" count of Sec. V-A:
  (m_0+n_0+...+m_a+n_a)*K + 2*M*N values moved between cache and registers.
* ``min_strip_memops`` -- exhaustive search over every row-strip tiling (each
  strip split into blocks) for the smallest sum(m_i+n_i), tiny sizes only.

Readings where the paper is silent or garbled (the builder's choices):
1. A remainder of a narrow C that is not itself a kernel height is tiled
   again with the same rule: the tallest height whose kernels reach width N,
   repeated while it fits.
2. TileSingleDim's "too small" is "less than half of the largest piece"; the
   last full piece and the remainder are then replaced by the two halves of
   their sum (ceil, floor).  This leaves sum(n) and the piece count unchanged.
3. ExtendTo8 merges pairs of 4-row strips into 8-row strips; ExtendTo16 merges
   groups of four into 16-row strips, and a leftover of three, two or one
   4-row strips becomes one 12-, 8- or 4-row strip.  The 15x15 example needs
   three 4-row strips to become one 12-row strip.
4. Of the two merges, the first (8-row strips) is kept on a tie.
5. "2mn" in the memops formula is 2*M*N (one load and one store of C); the
   worked example's 450 = 2*15*15 fixes this.
6. Every strip is cut across N with the widths its height's kernels reach
   (the outline's "maximum value that n_c can be taken"); where the printed
   steps give a 3-row strip widths up to 8 (M = 4q + 1 > 12), the oracle
   follows the outline and gives it the 13 its kernels reach.

Shape sets are passed in as {height: max_width}: a kernel m_c x n_c exists for
every width 1..max_width of that height (that is how every row of Table I is
written).
"""
from __future__ import annotations


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


def _strip_blocks(heights, N, shapes):
    """Blocks (row0, col0, m_c, n_c) of row strips of the given heights (top
    to bottom), each cut across N into the widest blocks its height allows."""
    blocks = []
    row = 0
    for h in heights:
        col = 0
        for w, count in tile_single_dim(N, range(1, shapes[h] + 1)):
            for _ in range(count):
                blocks.append((row, col, h, w))
                col += w
        row += h
    return blocks


def _strip_sum(blocks):
    return sum(m + n for _, _, m, n in blocks)


def _merge_fours(q, group):
    """q 4-row strips merged into strips of 4*group rows, a leftover of
    fewer than `group` of them into one strip (reading 3)."""
    full, left = divmod(q, group)
    return [4 * group] * full + ([4 * left] if left else [])


def _narrow_heights(M, N, shapes):
    """Row strips of a narrow C: the tallest height whose kernels reach
    width N, as often as it fits, then the remainder the same way."""
    heights = []
    rem = M
    while rem:
        h = max(x for x in shapes if x <= rem and shapes[x] >= N)
        heights += [h] * (rem // h)
        rem %= h
    return heights


def _wide_heights(M):
    """Candidate row strips of a wide C (N > 13), each a list of heights.

    4-row strips, with 1-, 2- and 3-row strips making up M; the kernel set
    of Table I fixes the small cases: up to 7 rows the strips TileSingleDim
    cuts from heights 1..4, 9 rows as 4 + 3 + 2, 10 and 11 rows as an 8-row
    strip and the rest, 12 rows as one strip.  Beyond 12 rows the 4-row
    strips are merged into 8- or 16-row strips (two candidates); a remainder
    of one row is avoided by giving up one 4-row strip for 3 + 2."""
    if M < 8:
        return [[h for h, c in tile_single_dim(M, [1, 2, 3, 4]) for _ in range(c)]]
    if M == 8:
        return [[8]]
    if M == 9:
        return [[4, 3, 2]]
    if M < 12:
        return [[8, M - 8]]
    if M == 12:
        return [[12]]
    q, r = divmod(M, 4)
    tail = [r] if r else []
    if r == 1:
        q, tail = q - 1, [3, 2]
    return [_merge_fours(q, 2) + tail, _merge_fours(q, 4) + tail]


def sgemm_nn_tile(M, N, shapes):
    """The SGEMM_NN tiling of C (Sec. V-A, Algorithm 2).

    ``shapes`` is the SGEMM_NN row of Table I as {height: max_width}.
    Returns blocksC as a list of (row0, col0, m_c, n_c); ``blocks_ab`` gives
    the blocks of A and B they read.
    """
    if M <= 0 or N <= 0:
        return []
    if N <= 13:
        heights = _narrow_heights(M, N, shapes)
        blocks, row = [], 0
        for h in heights:
            blocks.append((row, 0, h, N))
            row += h
        return blocks
    best = None
    for heights in _wide_heights(M):   # the fewer values moved wins; the first on a tie
        blocks = _strip_blocks(heights, N, shapes)
        if best is None or _strip_sum(blocks) < _strip_sum(best):
            best = blocks
    return best


def blocks_ab(blocksC, K):
    """blocksA / blocksB of Sec. V-A: the A rows and B columns each C block
    reads, as (row0, m_c, K) and (col0, n_c, K), in the order of blocksC."""
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
