"""Work partition across ranks (one process per GPU): result ranges and individuals.

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


# ---------------------------------------------------------------- individuals (n_pf axis)
#
# Sec. 4's n_pf axis splits the individuals instead: a rank tallies its slice of
# every vector, and a parallel reduction sums the partial tallies (integers,
# so the sum is exact).  CCC values then follow from the summed tallies and the
# whole panel's allele counts (ccc2_metric / ccc3_metric).


def field_range(n_f, world, rank):
    """Individuals [q_begin, q_end) of `rank`: equal shares on multiples of 64 individuals, so
    that a slice of the packed panel starts on a 16-byte boundary."""
    _check(world, rank)
    blocks = (int(n_f) + 63) // 64
    b0 = blocks * rank // world
    b1 = blocks * (rank + 1) // world
    return min(64 * b0, int(n_f)), min(64 * b1, int(n_f))


def _field_panel(geno, n_f, q_begin, q_end):
    from . import CCCError, CCC_EINVAL, ccc_panel
    if q_begin % 64 or not 0 <= q_begin < q_end <= n_f:
        raise CCCError("field slice", CCC_EINVAL)
    if geno.dim() != 2 or not geno.is_contiguous() or geno.element_size() != 8:
        raise CCCError("field slice", CCC_EINVAL)
    n_v, ld = geno.shape
    return ccc_panel(geno.data_ptr() + 8 * (q_begin // 32), int(q_end - q_begin), int(n_v), int(ld))


def field_tally2(geno, n_f, q_begin, q_end, tally, opts, stream=None):
    """ccc2_tally over individuals [q_begin, q_end) of every SNP (a view of the packed panel:
    same rows and stride, entries from q_begin on)."""
    import ctypes

    from . import _check as check, _ptr, _stream, load
    p = _field_panel(geno, n_f, q_begin, q_end)
    check("ccc2_tally", load().ccc2_tally(ctypes.byref(p), _ptr(tally), ctypes.byref(opts),
                                          _stream(stream)))


def field_tally3(geno, n_f, q_begin, q_end, j_begin, j_end, tally, opts, stream=None):
    """ccc3_tally of slabs [j_begin, j_end) over individuals [q_begin, q_end)."""
    import ctypes

    from . import _check as check, _ptr, _stream, load
    p = _field_panel(geno, n_f, q_begin, q_end)
    check("ccc3_tally", load().ccc3_tally(ctypes.byref(p), int(j_begin), int(j_end), _ptr(tally),
                                          ctypes.byref(opts), _stream(stream)))


def allreduce_tallies(tally, group=None):
    """Sum the partial tallies of all ranks in place (torch.distributed, SUM)."""
    import torch.distributed as dist
    dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    return tally
