"""The paper's 3-way route through masked matrices X_{j,xi} (Sec. 3.2).

TEST INFRASTRUCTURE ONLY (see :mod:`oracle`).  Used to cross-check the direct
3-way loop of the C oracle by a second, structurally different route:

1. for a fixed SNP column v_j, build three masked copies X_{j,1}, X_{j,2},
   X_{j,3} of the panel V following Table "Values of X_{j,xi}": column p of
   X_{j,xi} takes v_j's entry where V's entry in column p is (0,0), (0,1),
   (1,1) for xi = 1, 2, 3 respectively, and the null marker (1,0) otherwise;
2. form B_{j,xi} = X_{j,xi}^T o_3 V, the 2-way pairing tally that discards
   null entries of X (and, with missing data, missing entries of V, following
   Sec. 7 item 1 which reuses the skip for the missing marker);
3. reconstruct the 3-way table from the three 2-way tables:
       r_{ijk}(0,b,c) = 2 (B_{j,1})_{(i,k)}(b,c) + (B_{j,2})_{(i,k)}(b,c)
       r_{ijk}(1,b,c) = 2 (B_{j,3})_{(i,k)}(b,c) + (B_{j,2})_{(i,k)}(b,c)
   The paper writes f for these left-hand sides; they are read here as the
   integer tallies before the 1/(8 n_f) normalisation.  Index a belongs to
   SNP i (the column of V that selected the mask), b to v_j and c to v_k.

Entries are 2-bit codes 2*(v)_1 + (v)_2; the pairing tally of an X entry
x = (x_1, x_2) with a V entry y = (y_1, y_2) adds one to cell (x_r, y_s) for
each of the four choices r, s in {1, 2} (the enumeration of Fig. 1).
"""

from __future__ import annotations

import numpy as np

NULL = 0b10  # the (1,0) pair: null indicator in X, missing marker in V

# Table "Values of X_{j,xi}": (V entry, v_j entry) -> (X_{j,1}, X_{j,2}, X_{j,3}).
# (0,0)=0b00, (0,1)=0b01, (1,1)=0b11, null (1,0)=0b10.
XJC_TABLE = {
    (0b00, 0b00): (0b00, NULL, NULL),
    (0b00, 0b01): (0b01, NULL, NULL),
    (0b00, 0b11): (0b11, NULL, NULL),
    (0b01, 0b00): (NULL, 0b00, NULL),
    (0b01, 0b01): (NULL, 0b01, NULL),
    (0b01, 0b11): (NULL, 0b11, NULL),
    (0b11, 0b00): (NULL, NULL, 0b00),
    (0b11, 0b01): (NULL, NULL, 0b01),
    (0b11, 0b11): (NULL, NULL, 0b11),
}


def build_x(codes: np.ndarray, j: int):
    """X_{j,1..3} as code arrays [n_v, n_f] from the panel codes [n_v, n_f].

    A missing V entry or a missing v_j entry gives the null marker in all three.
    """
    n_v, n_f = codes.shape
    xs = [np.full((n_v, n_f), NULL, dtype=np.uint8) for _ in range(3)]
    vj = codes[j]
    for (v_code, j_code), triple in XJC_TABLE.items():
        sel = (codes == v_code) & (vj[None, :] == j_code)
        for xi in range(3):
            xs[xi][sel] = triple[xi]
    return xs


def _pairing_counts(codes: np.ndarray):
    """Per entry, how many of its two alleles equal 0 and 1; null/missing entries count nothing."""
    hi = (codes >> 1) & 1
    lo = codes & 1
    valid = codes != NULL
    c0 = ((hi == 0).astype(np.int64) + (lo == 0)) * valid
    c1 = ((hi == 1).astype(np.int64) + (lo == 1)) * valid
    return c0, c1


def tally_o3(x: np.ndarray, v: np.ndarray):
    """B = X^T o_3 V: for every column pair (i, k) the 2x2 pairing tally [n_v, n_v, 2, 2]."""
    x0, x1 = _pairing_counts(x)
    v0, v1 = _pairing_counts(v)
    xs = (x0, x1)
    vs = (v0, v1)
    n_v = x.shape[0]
    out = np.zeros((n_v, v.shape[0], 2, 2), dtype=np.int64)
    for b in range(2):
        for c in range(2):
            out[:, :, b, c] = xs[b] @ vs[c].T
    return out


def ccc3_tallies_slab(codes: np.ndarray, j: int):
    """All 3-way tallies r_{ijk}(a,b,c) for the slab of fixed j: array [n_v(i), n_v(k), 2, 2, 2]."""
    x1, x2, x3 = build_x(codes, j)
    b1 = tally_o3(x1, codes)
    b2 = tally_o3(x2, codes)
    b3 = tally_o3(x3, codes)
    n_v = codes.shape[0]
    r = np.zeros((n_v, n_v, 2, 2, 2), dtype=np.int64)
    r[:, :, 0] = 2 * b1 + b2
    r[:, :, 1] = 2 * b3 + b2
    return r


def ccc3_tallies(codes: np.ndarray):
    """Tallies for all triples i < j < k in slab order, [ntrip, 8] int64."""
    n_v = codes.shape[0]
    rows = []
    for j in range(n_v):
        r = ccc3_tallies_slab(codes, j)
        for i in range(j):
            for k in range(j + 1, n_v):
                rows.append(r[i, k].reshape(8))
    if not rows:
        return np.zeros((0, 8), np.int64)
    return np.stack(rows)
