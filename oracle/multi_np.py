"""Second oracle route for markers with s states: count matrices and one product.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Sec. 3.1 writes the
2-way tallies as a matrix product; with s states the count matrix of SNP i is
the s x n_f matrix of rho_{i,q}(a) (Sec. 2.1), and the s x s tally table of a
pair is the product of SNP i's matrix with SNP j's transposed.  This route
decodes every entry into those counts with array operations and forms the
products with a float64 matrix multiply (exact: every sum is an integer below
2^53); the direct per-individual loop of ``ccc_oracle_multi.c`` is the other
route.  CCC values follow Eqs. 1-3 over S = {0..s-1} with the same readings
for missing data (PERSNP / JOINT, n_ij = 0 -> 0).
"""

from __future__ import annotations

import numpy as np

NORM_PERSNP = 0
NORM_JOINT = 1


def decode(geno, n_f, s):
    """rho [n_v, s, n_f] (int64) and the non-missing mask m [n_v, n_f] (int64)."""
    g = np.asarray(geno, dtype=np.uint8)[:, :n_f]
    lo = (g & 15).astype(np.int64)
    hi = (g >> 4).astype(np.int64)
    present = (lo < s) & (hi < s)
    a = np.arange(s)[None, :, None]
    rho = (lo[:, None, :] == a).astype(np.int64) + (hi[:, None, :] == a).astype(np.int64)
    rho *= present[:, None, :]
    return rho, present.astype(np.int64)


def ccc2_multi_rows(geno, n_f, s, rows, gamma=2.0 / 3.0, norm=NORM_PERSNP):
    """Same contract as :func:`oracle.ccc2_multi_rows`."""
    rho, m = decode(geno, n_f, s)
    n_v = rho.shape[0]
    rf = rho.astype(np.float64)
    mf = m.astype(np.float64)
    s_counts = rho.sum(axis=2)  # [n_v, s]
    n_i = m.sum(axis=1)
    tallies, cccs = [], []
    for i in np.asarray(rows, dtype=np.int64):
        js = np.arange(i + 1, n_v)
        if js.size == 0:
            continue
        r = np.einsum("aq,jbq->jab", rf[i], rf[js])  # [J, s, s]
        r = np.rint(r).astype(np.int64)
        n_ij = np.rint(mf[js] @ mf[i]).astype(np.int64)  # jointly present count
        d = 4.0 * n_ij[:, None, None]
        with np.errstate(divide="ignore", invalid="ignore"):
            f = np.where(d > 0, r / d, 0.0)
            if norm == NORM_JOINT:
                fi = np.where(d[:, :, 0] > 0, r.sum(axis=2) / d[:, :, 0], 0.0)  # [J, s]
                fj = np.where(d[:, 0, :] > 0, r.sum(axis=1) / d[:, 0, :], 0.0)
            else:
                fi_row = np.where(n_i[i] > 0, s_counts[i] / (2.0 * max(n_i[i], 1)), 0.0)
                fi = np.broadcast_to(fi_row, (js.size, s))
                fj = np.where(n_i[js, None] > 0, s_counts[js] / (2.0 * np.maximum(n_i[js, None], 1)), 0.0)
        c = f * (1.0 - gamma * fi[:, :, None]) * (1.0 - gamma * fj[:, None, :])
        tallies.append(r.reshape(js.size, s * s))
        cccs.append(c.reshape(js.size, s * s))
    if not tallies:
        return np.zeros((0, s * s), np.int64), np.zeros((0, s * s), np.float64)
    return np.concatenate(tallies), np.concatenate(cccs)
