"""Pins of the oracle for markers with s allele states (Sec. 7 item 2 extension of Eqs. 1-3).

Each check ties the oracle to something other than its own code:

* hand-derived worked examples (``tests/golden/multi_hand_examples.json``);
* exhaustive enumeration of one individual (n_f = 1) over every entry value,
  against the definition rho(a) = [x == a] + [y == a] written out with exact
  fractions;
* the closed form of the analytic panel v_{i,q} = ((i + q) mod s, (i + 2q) mod s);
* the reduction s = 2 -> the biallelic oracle (pinned by tests/test_oracle.py);
* invariants: sum_ab r = 4 n_ij, sum_b r^{ab} = 2 sum_q rho_i(a) m_j, symmetry
  r_ij^{ab} = r_ji^{ba}, relabelling of states, PERSNP = JOINT without missing
  entries, frequencies summing to one;
* the second route (oracle/multi_np.py: decode + matrix product).
"""

import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import multi_np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "multi_hand_examples.json")
G = Fraction(2, 3)


def _panel(rows_hex, ld=16):
    out = np.zeros((len(rows_hex), ld), np.uint8)
    for i, row in enumerate(rows_hex):
        out[i, :len(row)] = [int(h, 16) for h in row]
    return out


@pytest.mark.parametrize("norm", [0, 1])
def test_golden_multi(norm):
    ex_all = json.load(open(GOLDEN))["examples"]
    for ex in ex_all:
        s = ex["s"]
        g = _panel(ex["snps"])
        n_f = len(ex["snps"][0])
        t, c = oracle.ccc2_multi_all(g, n_f, s, norm=norm)
        np.testing.assert_array_equal(t[0], ex["tally"], err_msg=ex["name"])
        want = [float(Fraction(x)) for x in ex["ccc_persnp" if norm == 0 else "ccc_joint"]]
        np.testing.assert_allclose(c[0], want, rtol=1e-15, atol=0, err_msg=ex["name"])


def _entries(s):
    """Every entry byte of one individual: the unordered state pairs and a missing value."""
    vals = [x | (y << 4) for x in range(s) for y in range(x, s)]
    # 0xFF, a byte whose low nibble is s and one whose high nibble is s: all missing
    return vals + [0xFF, s, s << 4]


def _rho(e, s):
    x, y = e & 15, e >> 4
    if x >= s or y >= s:
        return [0] * s
    return [int(x == a) + int(y == a) for a in range(s)]


@pytest.mark.parametrize("s", [2, 3, 4])
def test_exhaustive_one_individual(s):
    ents = _entries(s)
    pairs = list(itertools.product(ents, ents))
    g = np.zeros((2 * len(pairs), 16), np.uint8)
    for k, (ei, ej) in enumerate(pairs):
        g[2 * k, 0] = ei
        g[2 * k + 1, 0] = ej
    pi = np.arange(0, 2 * len(pairs), 2)
    for norm in (0, 1):
        t, c = oracle.ccc2_multi_pairs(g, 1, s, pi, pi + 1, norm=norm)
        for k, (ei, ej) in enumerate(pairs):
            ri, rj = _rho(ei, s), _rho(ej, s)
            want_t = [ri[a] * rj[b] for a in range(s) for b in range(s)]
            assert list(t[k]) == want_t, (ei, ej)
            present = sum(ri) == 2 and sum(rj) == 2
            if not present:
                assert np.all(c[k] == 0.0)
                continue
            fi = [Fraction(x, 2) for x in ri]
            fj = [Fraction(x, 2) for x in rj]
            want_c = [Fraction(ri[a] * rj[b], 4) * (1 - G * fi[a]) * (1 - G * fj[b])
                      for a in range(s) for b in range(s)]
            np.testing.assert_allclose(c[k], [float(x) for x in want_c], rtol=1e-15, atol=0)


@pytest.mark.parametrize("s", [3, 5, 7])
def test_closed_form_analytic_panel(s):
    """v_{i,q} = (x, y) = ((i + q) mod s, (i + 2q) mod s), n_f a multiple of s, s odd.

    Over one period of q every state occurs once as x and once as y, so
    r_ij^{ab} = (n_f/s) (2 [b = a + d] + [b = j + 2(a - i)] + [2(b - j) = a - i])
    (mod s, d = j - i): the x-x and y-y terms keep the offset d, the x_i-y_j term
    fixes q by x_i = a, the y_i-x_j term by y_i = a.
    """
    n_v, n_f = 9, 4 * s
    i_ = np.arange(n_v)[:, None]
    q = np.arange(n_f)[None, :]
    x = (i_ + q) % s
    y = (i_ + 2 * q) % s
    g = np.zeros((n_v, 16 * ((n_f + 15) // 16)), np.uint8)
    g[:, :n_f] = (x | (y << 4)).astype(np.uint8)
    t, c = oracle.ccc2_multi_all(g, n_f, s)
    per = n_f // s
    inv2 = pow(2, -1, s)
    k = 0
    for i in range(n_v):
        for j in range(i + 1, n_v):
            d = (j - i) % s
            want = np.zeros((s, s), np.int64)
            for a in range(s):
                for b in range(s):
                    want[a, b] = per * (2 * int(b == (a + d) % s) + int(b == (j + 2 * (a - i)) % s)
                                        + int(b == (j + (a - i) * inv2) % s))
            np.testing.assert_array_equal(t[k].reshape(s, s), want, err_msg=f"{i},{j}")
            # every state has frequency 1/s: CCC = r / (4 n_f) (1 - g/s)^2
            np.testing.assert_allclose(c[k], want.ravel() / (4.0 * n_f) * (1 - 2 / (3 * s)) ** 2,
                                       rtol=1e-15)
            k += 1


@pytest.mark.parametrize("norm", [0, 1])
def test_reduces_to_biallelic(norm):
    n_v, n_f = 70, 301
    words = synth.panel_hwe(n_v, n_f, seed=12, p_missing=0.05)
    g = synth.multi_from_biallelic(words, n_f)
    t2, c2 = oracle.ccc2_all(words, n_f, norm=norm)
    tm, cm = oracle.ccc2_multi_all(g, n_f, 2, norm=norm)
    np.testing.assert_array_equal(tm, t2)
    np.testing.assert_allclose(cm, c2, rtol=1e-14, atol=0)


def test_invariants():
    s, n_v, n_f = 5, 30, 257
    g = synth.panel_multi(n_v, n_f, s, seed=13, p_missing=0.1, pad_seed=3)
    t, c = oracle.ccc2_multi_all(g, n_f, s)
    rho, m = multi_np.decode(g, n_f, s)
    present = [[(g[i, q] & 15) < s and (g[i, q] >> 4) < s for q in range(n_f)] for i in range(n_v)]
    k = 0
    for i in range(n_v):
        for j in range(i + 1, n_v):
            r = t[k].reshape(s, s)
            n_ij = sum(present[i][q] and present[j][q] for q in range(n_f))
            assert r.sum() == 4 * n_ij
            # sum_b rho_j(b) = 2 for a present entry, 0 for a missing one
            for a in range(s):
                assert r[a].sum() == 2 * sum(int(rho[i, a, q]) for q in range(n_f) if present[j][q])
            k += 1
    # symmetry: swapping the two SNPs transposes the table
    pi, pj = np.array([0, 3, 7]), np.array([5, 9, 20])
    t_ab, _ = oracle.ccc2_multi_pairs(g, n_f, s, pi, pj)
    g_sw = g.copy()
    for a, b in zip(pi, pj):
        g_sw[[a, b]] = g_sw[[b, a]]
    t_ba, _ = oracle.ccc2_multi_pairs(g_sw, n_f, s, pi, pj)
    for u in range(3):
        np.testing.assert_array_equal(t_ab[u].reshape(s, s), t_ba[u].reshape(s, s).T)


def test_state_relabelling_permutes_tables():
    s, n_v, n_f = 4, 12, 199
    g = synth.panel_multi(n_v, n_f, s, seed=14, p_missing=0.05)
    perm = np.array([2, 0, 3, 1])  # state a of SNP 0 becomes perm[a]
    h = g.copy()
    lo, hi = h[0, :n_f] & 15, h[0, :n_f] >> 4
    ok = (lo < s) & (hi < s)
    h[0, :n_f] = np.where(ok, perm[np.minimum(lo, s - 1)] | (perm[np.minimum(hi, s - 1)] << 4),
                          h[0, :n_f])
    for norm in (0, 1):
        t, c = oracle.ccc2_multi_rows(g, n_f, s, [0], norm=norm)
        tp, cp = oracle.ccc2_multi_rows(h, n_f, s, [0], norm=norm)
        for k in range(n_v - 1):
            np.testing.assert_array_equal(tp[k].reshape(s, s)[perm], t[k].reshape(s, s))
            np.testing.assert_allclose(cp[k].reshape(s, s)[perm], c[k].reshape(s, s), rtol=1e-15)


def test_no_missing_norms_agree_and_frequencies_sum_to_one():
    s, n_v, n_f = 6, 20, 150
    g = synth.panel_multi(n_v, n_f, s, seed=15, p_missing=0.0)
    _, c0 = oracle.ccc2_multi_all(g, n_f, s, norm=0)
    _, c1 = oracle.ccc2_multi_all(g, n_f, s, norm=1)
    np.testing.assert_allclose(c0, c1, rtol=1e-13)
    cnt = oracle.multi_counts(g, n_f, s)
    np.testing.assert_array_equal(cnt[:, :s].sum(1), 2 * cnt[:, s])
    assert np.all(cnt[:, s] == n_f)


def test_numpy_route_agrees():
    for s, p in ((2, 0.0), (3, 0.2), (8, 0.05), (15, 0.02)):
        g = synth.panel_multi(25, 211, s, seed=16, p_missing=p, pad_seed=5)
        rows = np.array([0, 3, 24, 11])
        for norm in (0, 1):
            t, c = oracle.ccc2_multi_rows(g, 211, s, rows, norm=norm)
            t2, c2 = multi_np.ccc2_multi_rows(g, 211, s, rows, norm=norm)
            np.testing.assert_array_equal(t, t2)
            np.testing.assert_allclose(c, c2, rtol=1e-14, atol=0)


def test_all_missing_snp_and_degenerate_sizes():
    s, n_f = 3, 40
    g = synth.panel_multi(6, n_f, s, seed=17, p_missing=0.0)
    g[2, :n_f] = 0xFF
    t, c = oracle.ccc2_multi_all(g, n_f, s)
    idx = oracle.pair_index(np.array([0, 1, 2, 2, 2]), np.array([2, 2, 3, 4, 5]), 6)
    assert np.all(t[idx] == 0) and np.all(c[idx] == 0.0)
    t1, c1 = oracle.ccc2_multi_all(g[:1], n_f, s)
    assert t1.shape == (0, 9) and c1.shape == (0, 9)
