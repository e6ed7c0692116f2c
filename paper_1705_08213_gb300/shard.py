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

Block-circulant 2-way decomposition (Sec. 4, the n_pv axis): the vectors are
cut into one block per rank, and rank p computes only the block row
(p, p), (p, p + 1), ..., (p, p + h) (indices mod the rank count), a
block-circulant subset of the blocks that holds every unordered block pair
once.  A rank then holds only the h + 1 vector blocks of its block row (about
half the panel) instead of all of it; see :func:`circulant_plan`.
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


# ---------------------------------------------------------------- block-circulant (n_pv axis)


def vector_blocks(n_v, world):
    """Bounds of the `world` vector blocks: equal shares on multiples of 128 SNPs (whole
    tensor-core tiles), b[0] = 0 <= ... <= b[world] = n_v."""
    if world < 1:
        raise ValueError("need world >= 1")
    units = (int(n_v) + 127) // 128
    return [min(128 * (units * r // world), int(n_v)) for r in range(world)] + [int(n_v)]


def circulant_offsets(world, rank):
    """Block offsets d of `rank`'s block row: blocks (rank, rank + d mod world).  Every unordered
    pair of blocks, and every diagonal block, is in exactly one rank's row: d = 0 .. (world - 1)
    // 2, plus d = world / 2 for the first half of the ranks when world is even (the block pair
    {p, p + world / 2} would otherwise appear in two rows)."""
    _check(world, rank)
    ds = list(range(0, (world - 1) // 2 + 1))
    if world % 2 == 0 and world > 1 and rank < world // 2:
        ds.append(world // 2)
    return ds


def circulant_plan(n_v, world, rank):
    """What `rank` holds and computes under the block-circulant decomposition.

    Returns a dict with
      blocks: the vector blocks of its block row, (rank + d) mod world for d in
              :func:`circulant_offsets`, in that order;
      snps:   for every SNP of the local panel (the blocks' SNPs concatenated in that order),
              its global index;
      rows:   (0, n_p): the local rows to compute.  Rows [0, n_p) of the local panel pair each
              SNP i of the rank's own block with every later local SNP j: the diagonal block
              (i < j in block p) and every off-diagonal block of the row, nothing else.
    """
    import numpy as np
    b = vector_blocks(n_v, world)
    blocks = [(rank + d) % world for d in circulant_offsets(world, rank)]
    snps = np.concatenate([np.arange(b[q], b[q + 1], dtype=np.int64) for q in blocks]) \
        if blocks else np.zeros(0, np.int64)
    return {"blocks": blocks, "snps": snps, "rows": (0, b[rank + 1] - b[rank]),
            "n_v": int(n_v), "world": world, "rank": rank}


def circulant_local_panel(geno, plan):
    """The rank's local panel: the rows of its blocks (host numpy or device torch panel)."""
    return geno[plan["snps"]] if not hasattr(geno, "index_select") else \
        geno.index_select(0, _as_index(geno, plan["snps"]))


def _as_index(t, idx):
    import torch
    return torch.as_tensor(idx, dtype=torch.int64, device=t.device)


def circulant_pairs(plan):
    """Global indices (i < j) of the pairs of the rank's block row, in the local output order
    (rows [0, n_p) of the local panel, j increasing within a row), and a flag per pair that is
    True where the local pair is (j, i) globally, so that its 2 x 2 tables are transposed."""
    import numpy as np
    snps = plan["snps"]
    n_loc = snps.size
    n_p = plan["rows"][1]
    li = np.repeat(np.arange(n_p, dtype=np.int64), n_loc - 1 - np.arange(n_p, dtype=np.int64))
    starts = np.cumsum(np.concatenate([[0], n_loc - 1 - np.arange(n_p - 1, dtype=np.int64)]))
    lj = (np.arange(li.size, dtype=np.int64) - starts[li]) + li + 1 if li.size else li
    gi, gj = snps[li], snps[lj]
    swap = gi > gj
    lo, hi = np.where(swap, gj, gi), np.where(swap, gi, gj)
    return lo, hi, swap


def circulant_scatter(plan, tally, ccc=None):
    """Place the rank's block-row results in the global pair order.

    tally, ccc: the local outputs [pairs of rows (0, n_p)][4] (numpy).  Returns (global pair
    index, tally, ccc) with the tables of transposed pairs reordered (ab -> ba: entries 1 and 2
    swap), so that entry (a, b) refers to the allele a of the lower global index."""
    import numpy as np
    lo, hi, swap = circulant_pairs(plan)
    idx = lo * (2 * plan["n_v"] - lo - 1) // 2 + (hi - lo - 1)
    perm = np.array([0, 2, 1, 3])
    t = np.where(swap[:, None], tally[:, perm], tally)
    c = None if ccc is None else np.where(swap[:, None], ccc[:, perm], ccc)
    return idx, t, c


def circulant_block_row(geno_local, n_f, plan, tally, ccc, opts, stream=None):
    """The rank's block row on its GPU: ccc2_tally_metric_rows over rows (0, n_p) of the local
    panel (tally, ccc: device [ccc2_rows_count(n_local, 0, n_p)][4])."""
    from . import ccc2_tally_metric_rows
    lo, hi = plan["rows"]
    ccc2_tally_metric_rows(geno_local, n_f, lo, hi, tally, ccc, opts, stream)


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
