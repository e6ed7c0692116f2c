"""CPU oracle for the CCC tallies and metrics (Joubert et al., Secs. 2-3).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the CUDA path.  It shares no
code with the CUDA path.

Markers with s allele states (Sec. 7 item 2, the multi-allelic extension) have
:func:`multi_counts`, :func:`ccc2_multi_rows`, :func:`ccc2_multi_all` and
:func:`ccc2_multi_pairs` (C, ``oracle/ccc_oracle_multi.c``), cross-checked by the
numpy route :mod:`oracle.multi_np`.

Two routes are provided for biallelic SNPs:

* :mod:`oracle.ccc_oracle` (C, loaded here through ctypes) -- the direct
  definitions, Eqs. 1-5, one loop over individuals per pair or triple;
* :mod:`oracle.xjc` (numpy) -- the paper's own 3-way route through the masked
  matrices X_{j,xi} of Table "Values of X_{j,xi}" and the reconstruction
  formulas of Sec. 3.2, used to cross-check the direct 3-way loop.

Parity status: every function here is pinned by tests in ``tests/``
(brute-force enumeration, hand-derived examples in ``tests/golden/``, the
closed-form panel, invariants and exact rational arithmetic).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

NORM_PERSNP = 0
NORM_JOINT = 1
GAMMA = 2.0 / 3.0

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        f64p = ctypes.POINTER(ctypes.c_double)
        I64 = ctypes.c_int64
        lib.oracle_allele_counts.argtypes = [u64p, I64, I64, I64, i64p, i64p, i64p]
        lib.oracle_allele_counts.restype = None
        lib.oracle_ccc2_rows.argtypes = [u64p, I64, I64, I64, i64p, I64, ctypes.c_double,
                                         ctypes.c_int, i64p, f64p]
        lib.oracle_ccc2_rows.restype = ctypes.c_int
        lib.oracle_ccc2_pairs.argtypes = [u64p, I64, I64, I64, i64p, i64p, I64, ctypes.c_double,
                                          ctypes.c_int, i64p, f64p]
        lib.oracle_ccc2_pairs.restype = ctypes.c_int
        lib.oracle_ccc3_rows.argtypes = [u64p, I64, I64, I64, i64p, i64p, I64, ctypes.c_double,
                                         ctypes.c_int, i64p, f64p]
        lib.oracle_ccc3_rows.restype = ctypes.c_int
        lib.oracle_ccc3_triples.argtypes = [u64p, I64, I64, I64, i64p, i64p, i64p, I64,
                                            ctypes.c_double, ctypes.c_int, i64p, f64p]
        lib.oracle_ccc3_triples.restype = ctypes.c_int
        lib.oracle_threads.restype = ctypes.c_int
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.oracle_checksum.argtypes = [u32p, I64, I64, ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_checksum.restype = None
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.oracle_multi_counts.argtypes = [u8p, I64, I64, I64, ctypes.c_int, i64p]
        lib.oracle_multi_counts.restype = None
        lib.oracle_multi_rows.argtypes = [u8p, I64, I64, I64, ctypes.c_int, i64p, I64,
                                          ctypes.c_double, ctypes.c_int, i64p, f64p]
        lib.oracle_multi_rows.restype = ctypes.c_int
        lib.oracle_multi_pairs.argtypes = [u8p, I64, I64, I64, ctypes.c_int, i64p, i64p, I64,
                                           ctypes.c_double, ctypes.c_int, i64p, f64p]
        lib.oracle_multi_pairs.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _geno(geno):
    g = np.ascontiguousarray(geno, dtype=np.uint64)
    if g.ndim != 2:
        raise ValueError("geno must be [n_v, ld] uint64")
    return g


def threads() -> int:
    """Host threads the oracle's OpenMP loops use."""
    return int(_load().oracle_threads())


def allele_counts(geno, n_f):
    """Per SNP: s^0, s^1 (allele sums, Eq. 1 numerators) and n_i (non-missing count)."""
    g = _geno(geno)
    n_v, ld = g.shape
    s0 = np.zeros(n_v, np.int64)
    s1 = np.zeros(n_v, np.int64)
    npres = np.zeros(n_v, np.int64)
    _load().oracle_allele_counts(_p(g, ctypes.c_uint64), n_f, n_v, ld, _p(s0, ctypes.c_int64),
                                 _p(s1, ctypes.c_int64), _p(npres, ctypes.c_int64))
    return s0, s1, npres


def ccc2_rows(geno, n_f, rows, gamma=GAMMA, norm=NORM_PERSNP):
    """2-way tallies/CCC for every listed row i against all j > i (Eqs. 2-3).

    Returns (tally int64 [P, 4], ccc float64 [P, 4]) with P = sum(n_v - 1 - i),
    rows in the listed order and j increasing inside each row.
    """
    g = _geno(geno)
    n_v, ld = g.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= n_v):
        raise ValueError("row out of range")
    P = int(np.sum(n_v - 1 - rows)) if rows.size else 0
    tally = np.zeros((max(P, 1), 4), np.int64)
    ccc = np.zeros((max(P, 1), 4), np.float64)
    rc = _load().oracle_ccc2_rows(_p(g, ctypes.c_uint64), n_f, n_v, ld, _p(rows, ctypes.c_int64),
                                  rows.size, gamma, norm, _p(tally, ctypes.c_int64),
                                  _p(ccc, ctypes.c_double))
    if rc:
        raise MemoryError("oracle_ccc2_rows")
    return tally[:P], ccc[:P]


def ccc2_all(geno, n_f, gamma=GAMMA, norm=NORM_PERSNP):
    """All unique pairs i < j in the upper-triangle order of :func:`pair_index`."""
    n_v = np.asarray(geno).shape[0]
    return ccc2_rows(geno, n_f, np.arange(n_v), gamma, norm)


def ccc2_pairs(geno, n_f, pi, pj, gamma=GAMMA, norm=NORM_PERSNP):
    """2-way tallies/CCC for explicit pairs (pi[t] < pj[t])."""
    g = _geno(geno)
    n_v, ld = g.shape
    pi = np.ascontiguousarray(pi, dtype=np.int64)
    pj = np.ascontiguousarray(pj, dtype=np.int64)
    if not (np.all(pi < pj) and np.all(pi >= 0) and np.all(pj < n_v)):
        raise ValueError("pairs must satisfy 0 <= i < j < n_v")
    n = pi.size
    tally = np.zeros((max(n, 1), 4), np.int64)
    ccc = np.zeros((max(n, 1), 4), np.float64)
    rc = _load().oracle_ccc2_pairs(_p(g, ctypes.c_uint64), n_f, n_v, ld, _p(pi, ctypes.c_int64),
                                   _p(pj, ctypes.c_int64), n, gamma, norm,
                                   _p(tally, ctypes.c_int64), _p(ccc, ctypes.c_double))
    if rc:
        raise MemoryError("oracle_ccc2_pairs")
    return tally[:n], ccc[:n]


def ccc3_rows(geno, n_f, ri, rj, gamma=GAMMA, norm=NORM_PERSNP):
    """3-way tallies/CCC for every listed (i, j), i < j, against all k > j (Eqs. 4-5)."""
    g = _geno(geno)
    n_v, ld = g.shape
    ri = np.ascontiguousarray(ri, dtype=np.int64)
    rj = np.ascontiguousarray(rj, dtype=np.int64)
    if not (np.all(ri < rj) and np.all(ri >= 0) and np.all(rj < n_v)):
        raise ValueError("rows must satisfy 0 <= i < j < n_v")
    P = int(np.sum(n_v - 1 - rj)) if rj.size else 0
    tally = np.zeros((max(P, 1), 8), np.int64)
    ccc = np.zeros((max(P, 1), 8), np.float64)
    rc = _load().oracle_ccc3_rows(_p(g, ctypes.c_uint64), n_f, n_v, ld, _p(ri, ctypes.c_int64),
                                  _p(rj, ctypes.c_int64), ri.size, gamma, norm,
                                  _p(tally, ctypes.c_int64), _p(ccc, ctypes.c_double))
    if rc:
        raise MemoryError("oracle_ccc3_rows")
    return tally[:P], ccc[:P]


def slab_rows(n_v, j_begin, j_end):
    """The (i, j) rows of slabs j in [j_begin, j_end): slab-major j, then i < j."""
    ri, rj = [], []
    for j in range(j_begin, j_end):
        ri.append(np.arange(j, dtype=np.int64))
        rj.append(np.full(j, j, dtype=np.int64))
    if not ri:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(ri), np.concatenate(rj)


def ccc3_slabs(geno, n_f, j_begin=None, j_end=None, gamma=GAMMA, norm=NORM_PERSNP):
    """All triples i < j < k with j in [j_begin, j_end), in the slab order of :func:`triple_index`."""
    n_v = np.asarray(geno).shape[0]
    j_begin = 0 if j_begin is None else j_begin
    j_end = n_v if j_end is None else j_end
    ri, rj = slab_rows(n_v, j_begin, j_end)
    return ccc3_rows(geno, n_f, ri, rj, gamma, norm)


def ccc3_triples(geno, n_f, pi, pj, pk, gamma=GAMMA, norm=NORM_PERSNP):
    """3-way tallies/CCC for explicit triples (pi < pj < pk)."""
    g = _geno(geno)
    n_v, ld = g.shape
    pi, pj, pk = (np.ascontiguousarray(x, dtype=np.int64) for x in (pi, pj, pk))
    if not (np.all(pi < pj) and np.all(pj < pk) and np.all(pi >= 0) and np.all(pk < n_v)):
        raise ValueError("triples must satisfy 0 <= i < j < k < n_v")
    n = pi.size
    tally = np.zeros((max(n, 1), 8), np.int64)
    ccc = np.zeros((max(n, 1), 8), np.float64)
    rc = _load().oracle_ccc3_triples(_p(g, ctypes.c_uint64), n_f, n_v, ld, _p(pi, ctypes.c_int64),
                                     _p(pj, ctypes.c_int64), _p(pk, ctypes.c_int64), n, gamma,
                                     norm, _p(tally, ctypes.c_int64), _p(ccc, ctypes.c_double))
    if rc:
        raise MemoryError("oracle_ccc3_triples")
    return tally[:n], ccc[:n]


def pair_index(i, j, n_v):
    """Position of pair i < j in the row-major upper triangle (no diagonal)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return i * (2 * n_v - i - 1) // 2 + (j - i - 1)


def slab_offset(j, n_v):
    """Number of triples in slabs 0..j-1: sum_{j' < j} j' (n_v - 1 - j')."""
    j = np.asarray(j, dtype=np.int64)
    # sum j' (n_v-1) - sum j'^2 over j' < j
    s1 = (j - 1) * j // 2
    s2 = (j - 1) * j * (2 * j - 1) // 6
    return s1 * (n_v - 1) - s2


def triple_index(i, j, k, n_v):
    """Position of triple i < j < k in the slab order (j-major, then i, then k)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    k = np.asarray(k, dtype=np.int64)
    return slab_offset(j, n_v) + i * (n_v - 1 - j) + (k - j - 1)


# ---------------------------------------------------------------- markers with s states


def _multi_geno(geno, s):
    g = np.ascontiguousarray(geno, dtype=np.uint8)
    if g.ndim != 2:
        raise ValueError("geno must be [n_v, ld] uint8")
    if not 2 <= s <= 15:
        raise ValueError("s must be in [2, 15]")
    return g


def multi_counts(geno, n_f, s):
    """Per SNP: s_i^a for a < s (allele-state sums) and n_i (non-missing count): int64 [n_v, s+1]."""
    g = _multi_geno(geno, s)
    n_v, ld = g.shape
    out = np.zeros((n_v, s + 1), np.int64)
    _load().oracle_multi_counts(_p(g, ctypes.c_uint8), n_f, n_v, ld, s, _p(out, ctypes.c_int64))
    return out


def ccc2_multi_rows(geno, n_f, s, rows, gamma=GAMMA, norm=NORM_PERSNP):
    """Tallies and CCC of every listed row i against all j > i for markers with s states.

    Returns (tally int64 [P, s*s], ccc float64 [P, s*s]), P = sum(n_v - 1 - i), values
    (a, b) with a major, rows in the listed order and j increasing inside each row.
    """
    g = _multi_geno(geno, s)
    n_v, ld = g.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    P = int(np.sum(n_v - 1 - rows)) if rows.size else 0
    tally = np.zeros((max(P, 1), s * s), np.int64)
    ccc = np.zeros((max(P, 1), s * s), np.float64)
    rc = _load().oracle_multi_rows(_p(g, ctypes.c_uint8), n_f, n_v, ld, s, _p(rows, ctypes.c_int64),
                                   rows.size, gamma, norm, _p(tally, ctypes.c_int64),
                                   _p(ccc, ctypes.c_double))
    if rc == 1:
        raise ValueError("row out of range")
    if rc:
        raise MemoryError("oracle_multi_rows")
    return tally[:P], ccc[:P]


def ccc2_multi_all(geno, n_f, s, gamma=GAMMA, norm=NORM_PERSNP):
    """All unique pairs i < j in the order of :func:`pair_index`."""
    n_v = np.asarray(geno).shape[0]
    return ccc2_multi_rows(geno, n_f, s, np.arange(n_v), gamma, norm)


def ccc2_multi_pairs(geno, n_f, s, pi, pj, gamma=GAMMA, norm=NORM_PERSNP):
    """Tallies and CCC of explicit pairs pi[t] < pj[t] for markers with s states."""
    g = _multi_geno(geno, s)
    n_v, ld = g.shape
    pi = np.ascontiguousarray(pi, dtype=np.int64)
    pj = np.ascontiguousarray(pj, dtype=np.int64)
    if not (np.all(pi < pj) and np.all(pi >= 0) and np.all(pj < n_v)):
        raise ValueError("pairs must satisfy 0 <= i < j < n_v")
    n = pi.size
    tally = np.zeros((max(n, 1), s * s), np.int64)
    ccc = np.zeros((max(n, 1), s * s), np.float64)
    rc = _load().oracle_multi_pairs(_p(g, ctypes.c_uint8), n_f, n_v, ld, s, _p(pi, ctypes.c_int64),
                                    _p(pj, ctypes.c_int64), n, gamma, norm,
                                    _p(tally, ctypes.c_int64), _p(ccc, ctypes.c_double))
    if rc:
        raise MemoryError("oracle_multi_pairs")
    return tally[:n], ccc[:n]


def checksum(values, base=0):
    """Exact 128-bit checksum of an integer array's entries as 32-bit words (int64 tallies
    below 2^31 give the same words as the library's int32 output), global offset `base`."""
    v = np.asarray(values)
    if v.dtype == np.float32:
        w = np.ascontiguousarray(v).view(np.uint32).ravel()
    else:
        if v.size and (v.min() < 0 or v.max() >= 1 << 31):
            raise ValueError("tallies must lie in [0, 2^31)")
        w = np.ascontiguousarray(v.astype(np.uint32)).ravel()
    out = np.zeros(2, np.uint64)
    _load().oracle_checksum(_p(w, ctypes.c_uint32), w.size, int(base), _p(out, ctypes.c_uint64))
    return int(out[0]) | (int(out[1]) << 64)
