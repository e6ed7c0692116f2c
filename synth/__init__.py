"""Seeded synthetic genotype panels in the packed 2-bit format.

This module is shared by the CPU oracle's tests and by the CUDA path's tests and
benchmark.  It holds no part of the CCC arithmetic: it only draws genotypes and
packs/unpacks the storage format.

Storage format (the vector model of Sec. 2.1, with the missing-value marker of
Sec. 7 item 1):

* every entry ``v_{i,q}`` is a pair of allele bits ``((v)_1, (v)_2)``; it is
  stored as the 2-bit code ``2*(v)_1 + (v)_2``;
* genotype 0 (homozygous, allele pair (0,0)) -> code ``0b00``;
  genotype 1 (heterozygous, always stored as (0,1)) -> code ``0b01``;
  genotype 2 (homozygous, (1,1)) -> code ``0b11``;
  missing -> code ``0b10``, the pair (1,0) which the paper sets aside as the
  missing-entry marker;
* SNP ``i`` occupies uint64 words ``[i*ld, i*ld + ceil(n_f/32))``; entry ``q``
  sits at bits ``2*(q%32) .. 2*(q%32)+1`` of word ``q//32`` (LSB first);
  bits past ``n_f`` in the last word and words past ``ceil(n_f/32)`` are
  padding that every consumer must ignore.

Random numbers come from a counter-based SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), so that any
entry can be regenerated independently of all others:

    mix(z)            = the SplitMix64 finaliser (mix64 variant 13)
    G                 = 0x9E3779B97F4A7C15
    key(seed, p)      = mix(seed + (p+1)*G)                  per panel p
    key(seed, p, i)   = mix(key(seed, p) + (i+1)*G)          per SNP i
    u(p, i, q, t)     = mix(key(seed, p, i) + (2q + t + 1)*G)  t in {0, 1}
    u_maf(p, i)       = mix(key(seed, p, i) + 0)             per-SNP draw

Uniforms in [0,1) take the top 53 bits: ``(u >> 11) * 2**-53``.
Stream t=0 decides "missing", stream t=1 draws the genotype.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "CODE_HOM0", "CODE_HET", "CODE_MISSING", "CODE_HOM1", "MULTI_MISSING",
    "multi_state_thresholds", "genotypes_multi", "panel_multi", "multi_default_ld",
    "multi_from_biallelic",
    "mix64", "uniforms", "maf_beta_half", "genotypes_uniform", "genotypes_hwe",
    "genotypes_analytic", "codes_from_genotypes", "pack", "unpack", "words_per_snp", "fill_padding", "hwe_thresholds", "plant_near_duplicates",
    "panel_uniform", "panel_hwe", "panel_analytic", "default_ld",
]

CODE_HOM0 = 0b00
CODE_HET = 0b01
CODE_MISSING = 0b10
CODE_HOM1 = 0b11

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, panel: int, snps: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        kp = mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.uint64(panel + 1) * _G)
        return mix64(kp + (snps.astype(np.uint64) + np.uint64(1)) * _G)


def _to_unit(u: np.ndarray) -> np.ndarray:
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniforms(seed: int, panel: int, snps: np.ndarray, n_f: int, stream: int) -> np.ndarray:
    """u(p, i, q, t) for all listed SNPs and q in [0, n_f): float64 [len(snps), n_f]."""
    snps = np.asarray(snps, dtype=np.int64)
    k = _key(seed, panel, snps)[:, None]
    q = np.arange(n_f, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        ctr = k + (np.uint64(2) * q + np.uint64(stream + 1)) * _G
    return _to_unit(mix64(ctr))


def maf_beta_half(seed: int, panel: int, snps: np.ndarray) -> np.ndarray:
    """Per-SNP minor-allele frequency: Beta(1/2,1/2) folded to [0, 1/2], floored at 0.01.

    A Beta(1/2,1/2) variate is sin^2(pi*U/2) for U uniform on [0,1) (the arcsine
    law).  It is folded as p = min(x, 1-x) and then raised to at least 0.01.
    """
    snps = np.asarray(snps, dtype=np.int64)
    u = _to_unit(mix64(_key(seed, panel, snps)))
    x = np.sin(0.5 * np.pi * u) ** 2
    p = np.minimum(x, 1.0 - x)
    return np.maximum(p, 0.01)


def genotypes_uniform(seed, panel, snps, n_f, p_missing):
    """Genotype 0/1/2 uniform, missing i.i.d. with probability p_missing (-1 marks missing)."""
    um = uniforms(seed, panel, snps, n_f, 0)
    ug = uniforms(seed, panel, snps, n_f, 1)
    g = np.minimum((ug * 3.0).astype(np.int8), 2)
    g[um < p_missing] = -1
    return g


def genotypes_hwe(seed, panel, snps, n_f, p_missing):
    """Hardy-Weinberg genotypes: P(g) = (1-p)^2, 2p(1-p), p^2 with per-SNP p; -1 marks missing."""
    t0, t1 = hwe_thresholds(seed, panel, snps)
    t0, t1 = t0[:, None], t1[:, None]
    um = uniforms(seed, panel, snps, n_f, 0)
    ug = uniforms(seed, panel, snps, n_f, 1)
    g = np.where(ug < t0, 0, np.where(ug < t1, 1, 2)).astype(np.int8)
    g[um < p_missing] = -1
    return g


def genotypes_analytic(n_v, n_f):
    """The closed-form panel g_{i,q} = (i + q) mod 3, no missing entries."""
    i = np.arange(n_v)[:, None]
    q = np.arange(n_f)[None, :]
    return ((i + q) % 3).astype(np.int8)


_G2C = np.array([CODE_HOM0, CODE_HET, CODE_HOM1, CODE_MISSING], dtype=np.uint8)


def codes_from_genotypes(g: np.ndarray) -> np.ndarray:
    """Genotype array (0/1/2, -1 = missing) -> 2-bit codes (uint8 0..3)."""
    g = np.asarray(g)
    idx = np.where(g < 0, 3, g).astype(np.int64)
    return _G2C[idx]


def words_per_snp(n_f: int) -> int:
    return (n_f + 31) // 32


def default_ld(n_f: int) -> int:
    """Row stride in uint64 words: ceil(n_f/32) rounded up to an even count (16-byte rows)."""
    w = words_per_snp(n_f)
    return max(2, (w + 1) // 2 * 2)


def fill_padding(words: np.ndarray, n_f: int, pad_seed: int, row0: int = 0) -> None:
    """Overwrite the padding bits of packed rows with garbage (row index row0 + r).

    Padding = the bits past n_f in the last word and the words past ceil(n_f/32).
    """
    n_v, ld = words.shape
    w = words_per_snp(n_f)
    with np.errstate(over="ignore"):
        idx = (np.arange(n_v, dtype=np.uint64)[:, None] + np.uint64(row0)) * np.uint64(ld) \
            + np.arange(ld, dtype=np.uint64)[None, :]
        garbage = mix64(idx + np.uint64(pad_seed) * _G)
    tail = n_f - (w - 1) * 32
    if tail < 32:
        keep = np.uint64((1 << (2 * tail)) - 1)
        words[:, w - 1] = (words[:, w - 1] & keep) | (garbage[:, w - 1] & ~keep)
    if ld > w:
        words[:, w:] = garbage[:, w:]


def pack(codes: np.ndarray, ld: int | None = None, pad_seed: int | None = None,
         out: np.ndarray | None = None, row0: int = 0) -> np.ndarray:
    """Pack codes [n_v, n_f] (uint8 0..3) into uint64 words [n_v, ld].

    With ``pad_seed`` set, the padding bits (past n_f in the last word, and the
    words past ceil(n_f/32)) are filled with random garbage so that tests can
    check that consumers ignore them; otherwise they are zero.  ``out`` and
    ``row0`` let a caller pack a block of rows into a larger preallocated array
    (row0 also indexes the padding garbage).
    """
    codes = np.asarray(codes, dtype=np.uint8)
    n_v, n_f = codes.shape
    w = words_per_snp(n_f)
    if ld is None:
        ld = default_ld(n_f)
    if ld < w:
        raise ValueError("ld must be at least ceil(n_f/32)")
    padded = np.zeros((n_v, w * 32), dtype=np.uint8)
    padded[:, :n_f] = codes
    blk = padded.reshape(n_v, w, 32).astype(np.uint64)
    words = np.zeros((n_v, w), dtype=np.uint64)
    for k in range(32):
        words |= blk[:, :, k] << np.uint64(2 * k)
    if out is None:
        out = np.zeros((n_v, ld), dtype=np.uint64)
        dst = out
    else:
        dst = out[row0:row0 + n_v]
    dst[:, :w] = words
    if ld > w:
        dst[:, w:] = 0
    if pad_seed is not None:
        fill_padding(dst, n_f, pad_seed, row0)
    return out


def unpack(words: np.ndarray, n_f: int) -> np.ndarray:
    """Inverse of :func:`pack`: uint64 [n_v, ld] -> codes uint8 [n_v, n_f]."""
    words = np.asarray(words, dtype=np.uint64)
    n_v = words.shape[0]
    w = words_per_snp(n_f)
    out = np.empty((n_v, w, 32), dtype=np.uint8)
    for k in range(32):
        out[:, :, k] = ((words[:, :w] >> np.uint64(2 * k)) & np.uint64(3)).astype(np.uint8)
    return out.reshape(n_v, w * 32)[:, :n_f]


def _panel(gen, n_v, n_f, ld, pad_seed, chunk):
    if ld is None:
        ld = default_ld(n_f)
    out = np.zeros((n_v, ld), dtype=np.uint64)
    for r0 in range(0, n_v, chunk):
        r1 = min(n_v, r0 + chunk)
        g = gen(np.arange(r0, r1))
        pack(codes_from_genotypes(g), ld=ld, pad_seed=pad_seed, out=out, row0=r0)
    return out


_fast = None


def _fast_lib():
    """The C twin of the generators (synth/_gen.c), built on first use; None if unavailable."""
    global _fast
    if _fast is None:
        try:
            import ctypes

            from . import build as _b
            lib = ctypes.CDLL(_b.build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.synth_pack.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, dp, dp,
                                       ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]
            lib.synth_pack.restype = None
            lib.synth_multi.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_uint64, ctypes.c_int64, dp, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_uint8)]
            lib.synth_multi.restype = None
            _fast = lib
        except Exception:  # no compiler: the numpy definitions are used
            _fast = False
    return _fast or None


def _panel_fast(kind, n_v, n_f, ld, seed, panel, p_missing, pad_seed, t0=None, t1=None):
    import ctypes
    lib = _fast_lib()
    if ld is None:
        ld = default_ld(n_f)
    out = np.zeros((n_v, ld), dtype=np.uint64)
    dp = ctypes.POINTER(ctypes.c_double)
    a0 = None if t0 is None else np.ascontiguousarray(t0, dtype=np.float64)
    a1 = None if t1 is None else np.ascontiguousarray(t1, dtype=np.float64)
    lib.synth_pack(kind, n_v, n_f, ld, seed & 0xFFFFFFFFFFFFFFFF, panel, 0,
                   None if a0 is None else a0.ctypes.data_as(dp),
                   None if a1 is None else a1.ctypes.data_as(dp), float(p_missing),
                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    if pad_seed is not None:
        fill_padding(out, n_f, pad_seed)
    return out


def panel_uniform(n_v, n_f, seed=0, p_missing=0.02, panel=0, ld=None, pad_seed=None, fast=True):
    """Uniform-genotype panel (the small 2-way case): packed uint64 [n_v, ld]."""
    if fast and _fast_lib() is not None:
        return _panel_fast(0, n_v, n_f, ld, seed, panel, p_missing, pad_seed)
    chunk = max(1, (1 << 22) // max(n_f, 1))
    return _panel(lambda s: genotypes_uniform(seed, panel, s, n_f, p_missing), n_v, n_f, ld,
                  pad_seed, chunk)


def hwe_thresholds(seed, panel, snps):
    """Per-SNP genotype thresholds t0 = (1-p)^2, t1 = t0 + 2p(1-p) of the Hardy-Weinberg draw."""
    p = maf_beta_half(seed, panel, snps)
    t0 = (1.0 - p) ** 2
    return t0, t0 + 2.0 * p * (1.0 - p)


def panel_hwe(n_v, n_f, seed=1, p_missing=0.01, panel=0, ld=None, pad_seed=None, fast=True):
    """Hardy-Weinberg panel with Beta(1/2,1/2) minor-allele frequencies: packed uint64 [n_v, ld]."""
    if fast and _fast_lib() is not None:
        t0, t1 = hwe_thresholds(seed, panel, np.arange(n_v))
        return _panel_fast(1, n_v, n_f, ld, seed, panel, p_missing, pad_seed, t0, t1)
    chunk = max(1, (1 << 22) // max(n_f, 1))
    return _panel(lambda s: genotypes_hwe(seed, panel, s, n_f, p_missing), n_v, n_f, ld,
                  pad_seed, chunk)


def panel_analytic(n_v, n_f, ld=None):
    """Closed-form panel g_{i,q} = (i+q) mod 3 (no missing): packed uint64 [n_v, ld]."""
    return pack(codes_from_genotypes(genotypes_analytic(n_v, n_f)), ld=ld)


def plant_near_duplicates(geno: np.ndarray, n_f: int, n_pairs: int, seed: int, redraw: float = 0.01,
                          p_missing: float = 0.01):
    """Overwrite SNP rows with near-copies of other rows, in place.

    For each of ``n_pairs`` disjoint (source, target) pairs drawn with a seeded
    generator, the target row becomes a copy of the source row in which a
    fraction ``redraw`` of the entries is redrawn: genotype 0/1/2 with the
    source row's own genotype frequencies, missing with probability p_missing.
    Returns the (source, target) pairs as an int64 array [n_pairs, 2] with
    source < target or source > target as drawn.
    """
    n_v = geno.shape[0]
    rng = np.random.default_rng(seed)
    rows = rng.choice(n_v, size=2 * n_pairs, replace=False)
    pairs = rows.reshape(n_pairs, 2)
    for src, dst in pairs:
        codes = unpack(geno[src:src + 1], n_f)[0].copy()
        present = codes[codes != CODE_MISSING]
        freq = np.array([np.mean(present == c) for c in (CODE_HOM0, CODE_HET, CODE_HOM1)])
        freq = freq / freq.sum() if freq.sum() > 0 else np.full(3, 1 / 3)
        sel = rng.random(n_f) < redraw
        k = int(sel.sum())
        new = np.array([CODE_HOM0, CODE_HET, CODE_HOM1], np.uint8)[rng.choice(3, size=k, p=freq)]
        new[rng.random(k) < p_missing] = CODE_MISSING
        codes[sel] = new
        pack(codes[None, :], ld=geno.shape[1], out=geno, row0=dst)
    return pairs.astype(np.int64)


# ---------------------------------------------------------------- multi-allelic panels
#
# Markers with s allele states (the multi-allelic extension the paper sketches in
# Sec. 7 item 2): every entry is an unordered pair of states (x, y), x, y in {0..s-1},
# stored in one byte as x | (y << 4); an entry whose low or high nibble is >= s
# is missing, 0xFF being the value written here.  SNP i occupies bytes
# [i*ld, i*ld + n_f); bytes past n_f are padding that consumers must ignore.
#
# Draws (same SplitMix64 keys as above):
#   per-SNP state weights  x_a = sin^2(pi u_a / 2), u_a = unit(mix(k' + (a+1) G)),
#                          k' = mix(key(seed, p, i) ^ 0x5851F42D4C957F2D);
#                          p_a = max(x_a, 0.01) / sum_b max(x_b, 0.01)
#                          (Beta(1/2,1/2) weights floored at 0.01, normalised)
#   per entry              um = u(3q + 1), u1 = u(3q + 2), u2 = u(3q + 3) with
#                          u(c) = unit(mix(key(seed, p, i) + c G));
#                          missing if um < p_missing, else x = state of u1 and
#                          y = state of u2 under the cumulative weights
#                          (two alleles drawn independently: Hardy-Weinberg).

MULTI_MISSING = 0xFF
_MULTI_SALT = np.uint64(0x5851F42D4C957F2D)


def multi_default_ld(n_f: int) -> int:
    """Row stride in bytes of a multi-allelic panel: n_f rounded up to 16."""
    return max(16, (n_f + 15) // 16 * 16)


def multi_state_thresholds(seed, panel, snps, s):
    """Cumulative state weights c[r, a] = p_0 + .. + p_a of each listed SNP: float64 [len, s]."""
    snps = np.asarray(snps, dtype=np.int64)
    with np.errstate(over="ignore"):
        k2 = mix64(_key(seed, panel, snps) ^ _MULTI_SALT)[:, None]
        a = np.arange(s, dtype=np.uint64)[None, :]
        u = _to_unit(mix64(k2 + (a + np.uint64(1)) * _G))
    x = np.maximum(np.sin(0.5 * np.pi * u) ** 2, 0.01)
    c = np.cumsum(x / x.sum(axis=1, keepdims=True), axis=1)
    c[:, -1] = 1.0
    return c


def _entry_uniforms(seed, panel, snps, n_f, t):
    snps = np.asarray(snps, dtype=np.int64)
    k = _key(seed, panel, snps)[:, None]
    q = np.arange(n_f, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        return _to_unit(mix64(k + (np.uint64(3) * q + np.uint64(t + 1)) * _G))


def genotypes_multi(seed, panel, snps, n_f, s, p_missing):
    """Entry bytes x | (y << 4) of the listed SNPs (0xFF = missing): uint8 [len, n_f]."""
    c = multi_state_thresholds(seed, panel, snps, s)
    um = _entry_uniforms(seed, panel, snps, n_f, 0)
    out = []
    for t in (1, 2):
        u = _entry_uniforms(seed, panel, snps, n_f, t)
        st = (u[:, :, None] >= c[:, None, :]).sum(axis=2)
        out.append(np.minimum(st, s - 1).astype(np.uint8))
    g = out[0] | (out[1] << np.uint8(4))
    g[um < p_missing] = MULTI_MISSING
    return g


def _multi_fill_padding(rows, n_f, pad_seed, row0=0):
    n_v, ld = rows.shape
    if ld <= n_f:
        return
    with np.errstate(over="ignore"):
        idx = (np.arange(n_v, dtype=np.uint64)[:, None] + np.uint64(row0)) * np.uint64(ld) \
            + np.arange(n_f, ld, dtype=np.uint64)[None, :]
        rows[:, n_f:] = (mix64(idx + np.uint64(pad_seed) * _G) & np.uint64(0xFF)).astype(np.uint8)


def panel_multi(n_v, n_f, s, seed=6, p_missing=0.01, panel=0, ld=None, pad_seed=None, fast=True):
    """Multi-allelic panel with s states: uint8 [n_v, ld] (layout above)."""
    if not 2 <= s <= 15:
        raise ValueError("s must be in [2, 15]")
    if ld is None:
        ld = multi_default_ld(n_f)
    if ld < n_f:
        raise ValueError("ld must be at least n_f")
    out = np.zeros((n_v, ld), dtype=np.uint8)
    lib = _fast_lib() if fast else None
    if lib is not None:
        import ctypes
        c = np.ascontiguousarray(multi_state_thresholds(seed, panel, np.arange(n_v), s))
        lib.synth_multi(n_v, n_f, ld, s, seed & 0xFFFFFFFFFFFFFFFF, panel,
                        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(p_missing),
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    else:
        chunk = max(1, (1 << 21) // max(n_f, 1))
        for r0 in range(0, n_v, chunk):
            r1 = min(n_v, r0 + chunk)
            out[r0:r1, :n_f] = genotypes_multi(seed, panel, np.arange(r0, r1), n_f, s, p_missing)
    if pad_seed is not None:
        _multi_fill_padding(out, n_f, pad_seed)
    return out


def multi_from_biallelic(words, n_f, ld=None):
    """A packed 2-bit panel as a 2-state multi-allelic panel: 00 -> (0,0), 01 -> (0,1),
    11 -> (1,1), 10 (missing) -> 0xFF."""
    codes = unpack(words, n_f)
    lut = np.array([0x00, 0x10, MULTI_MISSING, 0x11], dtype=np.uint8)
    if ld is None:
        ld = multi_default_ld(n_f)
    out = np.zeros((codes.shape[0], ld), dtype=np.uint8)
    out[:, :n_f] = lut[codes]
    return out
