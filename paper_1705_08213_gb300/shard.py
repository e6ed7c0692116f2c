"""Work partition across ranks (one process per GPU).

Sec. 4 spreads the 2-way pairs (blocks of the triangle) and the 3-way triples
(slabs of fixed j) over processors; the blocks are independent, so no results
are exchanged.  Here every rank holds the whole panel and takes one contiguous
range, balanced by work:

* 2-way: rows [i_begin, i_end) of the triangle (pairs i < j with i in the
  range), from ``ccc2_phase_bounds`` (bounds on multiples of 64 SNPs);
* 3-way: slabs [j_begin, j_end), from ``ccc3_phase_bounds``;
* markers with s states: rows on multiples of a 256-row operand block, from
  ``ccc2_multi_phase_bounds``.

The ranges of all ranks cover the triangle (tetrahedron) exactly once, and a
rank's results form one contiguous block of the global output order, starting
at :func:`pair_offset` (:func:`triple_offset`).  The bound helpers are
host-only library calls and need no GPU.
"""

from __future__ import annotations

from . import (ccc2_count, ccc2_index, ccc2_multi_phase_bounds, ccc2_phase_bounds, ccc3_count,
               ccc3_phase_bounds)


def _check(world, rank):
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")


def pair_range(n_v, world, rank):
    """Rows [i_begin, i_end) of the 2-way triangle for `rank` of `world`."""
    _check(world, rank)
    if world == 1:
        return 0, int(n_v)
    b = ccc2_phase_bounds(n_v, world)
    return b[rank], b[rank + 1]


def multi_pair_range(n_v, s, world, rank):
    """Rows [i_begin, i_end) of the multi-allelic 2-way triangle (s states)."""
    _check(world, rank)
    if world == 1:
        return 0, int(n_v)
    b = ccc2_multi_phase_bounds(n_v, s, world)
    return b[rank], b[rank + 1]


def slab_range(n_v, world, rank):
    """Slabs [j_begin, j_end) of the 3-way tetrahedron for `rank` of `world`."""
    _check(world, rank)
    if world == 1:
        return 0, int(n_v)
    b = ccc3_phase_bounds(n_v, world)
    return b[rank], b[rank + 1]


def pair_offset(n_v, i_begin):
    """Global index of the first pair of rows starting at i_begin (the pair count of
    rows [0, i_begin))."""
    return ccc2_count(n_v) if i_begin >= n_v - 1 else ccc2_index(i_begin, i_begin + 1, n_v)


def triple_offset(n_v, j_begin):
    """Global index of the first triple of slabs starting at j_begin."""
    return ccc3_count(n_v, 0, j_begin)
