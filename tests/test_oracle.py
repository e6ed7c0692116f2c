"""Pins for the CPU oracle: values it must reproduce that do not come from itself.

* brute-force enumeration of allele pairings at n_f = 1 (the tally process of
  Figs. 1 and 2, Sec. 2) over every code pair / code triple;
* hand-derived worked examples (``tests/golden/hand_examples.json``);
* the closed-form panel g_{i,q} = (i+q) mod 3 (the analytically verifiable
  synthetic case of Sec. 5);
* invariants: tallies sum to 4 n_ij (8 n_ijk), symmetry in i and j, marginals
  reproduce the per-SNP allele sums, 3-way tallies marginalise to 2-way ones;
* the paper's second 3-way route through X_{j,xi} and B_{j,xi} (Sec. 3.2);
* exact rational evaluation of Eqs. 1-5 for the floating-point CCC values.
"""

import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import xjc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")
CODES = (0b00, 0b01, 0b10, 0b11)


def _panel_from_code_strings(snps):
    codes = np.array([[int(c, 2) for c in row] for row in snps], dtype=np.uint8)
    return synth.pack(codes, pad_seed=99), codes.shape[1]


def _pairings(code):
    """The two alleles of a code as listed in the entry; None for the missing marker (1,0)."""
    if code == 0b10:
        return None
    return ((code >> 1) & 1, code & 1)


# ---------------------------------------------------------------- brute force

def test_bruteforce_2way_all_code_pairs():
    """Fig. 1: enumerate the four pairings of the two entries and tally each (x, y) cell."""
    for ci, cj in itertools.product(CODES, CODES):
        geno = synth.pack(np.array([[ci], [cj]], np.uint8))
        tally, _ = oracle.ccc2_all(geno, 1)
        expect = np.zeros((2, 2), np.int64)
        pi, pj = _pairings(ci), _pairings(cj)
        if pi is not None and pj is not None:
            for x in pi:
                for y in pj:
                    expect[x, y] += 1
        np.testing.assert_array_equal(tally[0], expect.reshape(4), err_msg=f"{ci:02b} {cj:02b}")


def test_bruteforce_3way_all_code_triples():
    """Fig. 2: enumerate the eight combinations of the three entries and tally each cell."""
    for ci, cj, ck in itertools.product(CODES, CODES, CODES):
        geno = synth.pack(np.array([[ci], [cj], [ck]], np.uint8))
        tally, _ = oracle.ccc3_slabs(geno, 1)
        expect = np.zeros((2, 2, 2), np.int64)
        ps = [_pairings(c) for c in (ci, cj, ck)]
        if all(p is not None for p in ps):
            for x in ps[0]:
                for y in ps[1]:
                    for z in ps[2]:
                        expect[x, y, z] += 1
        np.testing.assert_array_equal(tally[0], expect.reshape(8))


def test_bruteforce_multi_entry_sums():
    """For n_f > 1 the per-entry tables are summed (Sec. 2.1): check on a random panel."""
    rng = np.random.default_rng(1)
    codes = rng.integers(0, 4, size=(5, 77), dtype=np.uint8)
    geno = synth.pack(codes, pad_seed=4)
    tally, _ = oracle.ccc2_all(geno, 77)
    t = 0
    for i in range(5):
        for j in range(i + 1, 5):
            expect = np.zeros((2, 2), np.int64)
            for q in range(77):
                pi, pj = _pairings(codes[i, q]), _pairings(codes[j, q])
                if pi is None or pj is None:
                    continue
                for x in pi:
                    for y in pj:
                        expect[x, y] += 1
            np.testing.assert_array_equal(tally[t], expect.reshape(4))
            t += 1


# ---------------------------------------------------------------- golden

def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("norm", [oracle.NORM_PERSNP, oracle.NORM_JOINT])
def test_golden_2way(norm):
    key = "ccc_persnp" if norm == oracle.NORM_PERSNP else "ccc_joint"
    for ex in _golden()["two_way"]:
        geno, n_f = _panel_from_code_strings(ex["snps"])
        tally, ccc = oracle.ccc2_all(geno, n_f, norm=norm)
        np.testing.assert_array_equal(tally[0], ex["tally"], err_msg=ex["name"])
        expect = np.array([float(Fraction(v)) for v in ex[key]])
        np.testing.assert_allclose(ccc[0], expect, rtol=1e-15, atol=0, err_msg=ex["name"])
        s0, s1, npres = oracle.allele_counts(geno, n_f)
        fi = [Fraction(int(s), 2 * int(npres[0])) if npres[0] else Fraction(0) for s in (s0[0], s1[0])]
        fj = [Fraction(int(s), 2 * int(npres[1])) if npres[1] else Fraction(0) for s in (s0[1], s1[1])]
        assert fi == [Fraction(v) for v in ex["f_i"]], ex["name"]
        assert fj == [Fraction(v) for v in ex["f_j"]], ex["name"]


@pytest.mark.parametrize("norm", [oracle.NORM_PERSNP, oracle.NORM_JOINT])
def test_golden_3way(norm):
    key = "ccc_persnp" if norm == oracle.NORM_PERSNP else "ccc_joint"
    for ex in _golden()["three_way"]:
        geno, n_f = _panel_from_code_strings(ex["snps"])
        tally, ccc = oracle.ccc3_slabs(geno, n_f, norm=norm)
        np.testing.assert_array_equal(tally[0], ex["tally"], err_msg=ex["name"])
        expect = np.array([float(Fraction(v)) for v in ex[key]])
        np.testing.assert_allclose(ccc[0], expect, rtol=1e-15, atol=0, err_msg=ex["name"])


# ---------------------------------------------------------------- closed form

RHO_OF_GENOTYPE = {0: (2, 0), 1: (1, 1), 2: (0, 2)}


def test_closed_form_panel_2way():
    """g_{i,q} = (i+q) mod 3 with n_f = 0 mod 3: every residue class of q occurs n_f/3 times,
    so r_ij^{ab} = (n_f/3) sum_t rho(t)(a) rho((t+j-i) mod 3)(b)."""
    n_v, n_f = 9, 300
    geno = synth.panel_analytic(n_v, n_f)
    tally, ccc = oracle.ccc2_all(geno, n_f)
    t = 0
    for i in range(n_v):
        for j in range(i + 1, n_v):
            expect = np.zeros((2, 2), np.int64)
            for g in range(3):
                gj = (g + j - i) % 3
                for a in range(2):
                    for b in range(2):
                        expect[a, b] += RHO_OF_GENOTYPE[g][a] * RHO_OF_GENOTYPE[gj][b]
            np.testing.assert_array_equal(tally[t], (n_f // 3) * expect.reshape(4))
            # every SNP has f_i = (1/2, 1/2): CCC = r/(4 n_f) * (2/3)^2
            np.testing.assert_allclose(ccc[t], tally[t] / (4 * n_f) * (4 / 9), rtol=1e-14)
            t += 1


def test_closed_form_panel_3way():
    n_v, n_f = 6, 30
    geno = synth.panel_analytic(n_v, n_f)
    tally, _ = oracle.ccc3_slabs(geno, n_f)
    t = 0
    for j in range(n_v):
        for i in range(j):
            for k in range(j + 1, n_v):
                expect = np.zeros((2, 2, 2), np.int64)
                for g in range(3):
                    gj, gk = (g + j - i) % 3, (g + k - i) % 3
                    for a, b, c in itertools.product(range(2), repeat=3):
                        expect[a, b, c] += (RHO_OF_GENOTYPE[g][a] * RHO_OF_GENOTYPE[gj][b]
                                            * RHO_OF_GENOTYPE[gk][c])
                np.testing.assert_array_equal(tally[t], (n_f // 3) * expect.reshape(8))
                t += 1


# ---------------------------------------------------------------- invariants

def _rho_m(codes):
    hi = (codes >> 1) & 1
    lo = codes & 1
    m = (codes != 0b10).astype(np.int64)
    r0 = ((hi == 0).astype(np.int64) + (lo == 0)) * m
    r1 = ((hi == 1).astype(np.int64) + (lo == 1)) * m
    return r0, r1, m


@pytest.fixture(scope="module")
def random_panel():
    n_v, n_f = 23, 171
    geno = synth.panel_uniform(n_v, n_f, seed=12, p_missing=0.15, pad_seed=5)
    return geno, n_f, synth.unpack(geno, n_f)


def test_allele_counts_invariants(random_panel):
    geno, n_f, codes = random_panel
    s0, s1, npres = oracle.allele_counts(geno, n_f)
    r0, r1, m = _rho_m(codes)
    np.testing.assert_array_equal(npres, m.sum(1))
    np.testing.assert_array_equal(s0 + s1, 2 * npres)  # f_i(0) + f_i(1) = 1 (Eq. 1)
    np.testing.assert_array_equal(s1, r1.sum(1))


def test_2way_invariants(random_panel):
    geno, n_f, codes = random_panel
    n_v = codes.shape[0]
    tally, ccc = oracle.ccc2_all(geno, n_f)
    _, r1, m = _rho_m(codes)
    r0 = 2 * m - r1
    rho = (r0, r1)
    t = 0
    for i in range(n_v):
        for j in range(i + 1, n_v):
            tab = tally[t].reshape(2, 2)
            n_ij = int(np.sum(m[i] * m[j]))
            assert tab.sum() == 4 * n_ij  # sum_ab f_ij = 1 (Eq. 2)
            for a in range(2):
                # row marginal: sum_b r^{ab} = 2 sum_q rho_i(a) m_j
                assert tab[a].sum() == 2 * np.sum(rho[a][i] * m[j])
            for b in range(2):
                assert tab[:, b].sum() == 2 * np.sum(m[i] * rho[b][j])
            t += 1
    # symmetry in i and j: reversing the SNP order transposes every table
    rev = np.ascontiguousarray(geno[::-1])
    tally_r, ccc_r = oracle.ccc2_all(rev, n_f)
    for i in range(n_v):
        for j in range(i + 1, n_v):
            a = oracle.pair_index(i, j, n_v)
            b = oracle.pair_index(n_v - 1 - j, n_v - 1 - i, n_v)
            np.testing.assert_array_equal(tally[a].reshape(2, 2), tally_r[b].reshape(2, 2).T)
            np.testing.assert_allclose(ccc[a].reshape(2, 2), ccc_r[b].reshape(2, 2).T, rtol=1e-15)


def test_no_missing_marginal_equals_allele_sums():
    geno = synth.panel_uniform(12, 200, seed=3, p_missing=0.0)
    tally, _ = oracle.ccc2_all(geno, 200)
    s0, s1, npres = oracle.allele_counts(geno, 200)
    assert np.all(npres == 200)
    t = 0
    for i in range(12):
        for j in range(i + 1, 12):
            tab = tally[t].reshape(2, 2)
            assert tab[0].sum() == 2 * s0[i] and tab[1].sum() == 2 * s1[i]
            assert tab[:, 0].sum() == 2 * s0[j] and tab[:, 1].sum() == 2 * s1[j]
            t += 1


def test_3way_invariants(random_panel):
    geno, n_f, codes = random_panel
    geno = np.ascontiguousarray(geno[:11])
    codes = codes[:11]
    n_v = 11
    tally, _ = oracle.ccc3_slabs(geno, n_f)
    t2, _ = oracle.ccc2_all(geno, n_f)
    _, r1, m = _rho_m(codes)
    rho = (2 * m - r1, r1)
    for j in range(n_v):
        for i in range(j):
            for k in range(j + 1, n_v):
                tab = tally[oracle.triple_index(i, j, k, n_v)].reshape(2, 2, 2)
                assert tab.sum() == 8 * int(np.sum(m[i] * m[j] * m[k]))
                for a in range(2):
                    for b in range(2):
                        # sum_c r^{abc} = 2 sum_q rho_i(a) rho_j(b) m_k
                        assert tab[a, b].sum() == 2 * np.sum(rho[a][i] * rho[b][j] * m[k])
    # with no missing data the 3-way tables marginalise to the 2-way ones
    geno_c = synth.panel_uniform(8, 90, seed=4, p_missing=0.0)
    t3, _ = oracle.ccc3_slabs(geno_c, 90)
    t2, _ = oracle.ccc2_all(geno_c, 90)
    for j in range(8):
        for i in range(j):
            for k in range(j + 1, 8):
                tab = t3[oracle.triple_index(i, j, k, 8)].reshape(2, 2, 2)
                np.testing.assert_array_equal(tab.sum(2), 2 * t2[oracle.pair_index(i, j, 8)].reshape(2, 2))
                np.testing.assert_array_equal(tab.sum(0), 2 * t2[oracle.pair_index(j, k, 8)].reshape(2, 2))
                np.testing.assert_array_equal(tab.sum(1), 2 * t2[oracle.pair_index(i, k, 8)].reshape(2, 2))


def test_3way_permutation_symmetry():
    geno = synth.panel_uniform(7, 64, seed=21, p_missing=0.1)
    tally, ccc = oracle.ccc3_slabs(geno, 64)
    perm = np.array([3, 0, 6, 1, 5, 2, 4])  # new SNP s is old SNP perm[s]
    tp, cp = oracle.ccc3_slabs(np.ascontiguousarray(geno[perm]), 64)
    inv = np.argsort(perm)
    for i, j, k in itertools.combinations(range(7), 3):
        new = sorted([(inv[i], 0), (inv[j], 1), (inv[k], 2)])
        order = [axis for _, axis in new]
        a = tally[oracle.triple_index(i, j, k, 7)].reshape(2, 2, 2)
        b = tp[oracle.triple_index(*[s for s, _ in new], 7)].reshape(2, 2, 2)
        np.testing.assert_array_equal(np.transpose(a, order), b)
        ca = ccc[oracle.triple_index(i, j, k, 7)].reshape(2, 2, 2)
        cb = cp[oracle.triple_index(*[s for s, _ in new], 7)].reshape(2, 2, 2)
        np.testing.assert_allclose(np.transpose(ca, order), cb, rtol=1e-14)


# ---------------------------------------------------------------- second 3-way route

def test_3way_direct_matches_xjc_route(random_panel):
    geno, n_f, codes = random_panel
    n = 10
    direct, _ = oracle.ccc3_slabs(np.ascontiguousarray(geno[:n]), n_f)
    via_x = xjc.ccc3_tallies(codes[:n])
    np.testing.assert_array_equal(direct, via_x)


def test_xjc_table_matches_rho_products():
    # every row of the table, at n_f = 1, reproduces the direct 3-way tally
    for ci, cj, ck in itertools.product((0, 1, 3), repeat=3):
        codes = np.array([[ci], [cj], [ck]], np.uint8)
        r = xjc.ccc3_tallies_slab(codes, 1)[0, 2].reshape(8)
        direct, _ = oracle.ccc3_slabs(synth.pack(codes), 1)
        np.testing.assert_array_equal(r, direct[0])


# ---------------------------------------------------------------- exact arithmetic for CCC

def _exact_ccc2(codes, i, j, gamma, joint):
    _, r1, m = _rho_m(codes)
    rho = (2 * m - r1, r1)
    n_ij = int(np.sum(m[i] * m[j]))
    r = [[int(np.sum(rho[a][i] * rho[b][j])) for b in range(2)] for a in range(2)]
    if n_ij == 0:
        return [Fraction(0)] * 4
    if joint:
        fi = [Fraction(r[a][0] + r[a][1], 4 * n_ij) for a in range(2)]
        fj = [Fraction(r[0][b] + r[1][b], 4 * n_ij) for b in range(2)]
    else:
        ni, nj = int(m[i].sum()), int(m[j].sum())
        fi = [Fraction(int(rho[a][i].sum()), 2 * ni) for a in range(2)]
        fj = [Fraction(int(rho[b][j].sum()), 2 * nj) for b in range(2)]
    return [Fraction(r[a][b], 4 * n_ij) * (1 - gamma * fi[a]) * (1 - gamma * fj[b])
            for a in range(2) for b in range(2)]


@pytest.mark.parametrize("norm", [oracle.NORM_PERSNP, oracle.NORM_JOINT])
def test_ccc2_exact_rational(random_panel, norm):
    geno, n_f, codes = random_panel
    _, ccc = oracle.ccc2_all(geno, n_f, gamma=2.0 / 3.0, norm=norm)
    g = Fraction(2, 3)
    n_v = codes.shape[0]
    for i in range(0, n_v, 3):
        for j in range(i + 1, n_v, 2):
            exact = _exact_ccc2(codes, i, j, g, norm == oracle.NORM_JOINT)
            got = ccc[oracle.pair_index(i, j, n_v)]
            for x, e in zip(got, exact):
                assert abs(Fraction(x) - e) <= Fraction(1, 10**14) * (abs(e) + Fraction(1, 10**30))


def test_gamma_parameter():
    """gamma enters only through the factors (1 - gamma f): gamma = 0 gives CCC = f_ij."""
    geno = synth.panel_uniform(6, 50, seed=2, p_missing=0.05)
    tally, ccc = oracle.ccc2_all(geno, 50, gamma=0.0)
    n_ij = tally.sum(1, keepdims=True) / 4
    np.testing.assert_allclose(ccc, np.where(n_ij > 0, tally / (4 * np.maximum(n_ij, 1)), 0), rtol=1e-15)


# ---------------------------------------------------------------- indexing and sampling

def test_pair_and_triple_index_enumerate_in_order():
    n_v = 13
    idx = [oracle.pair_index(i, j, n_v) for i in range(n_v) for j in range(i + 1, n_v)]
    assert idx == list(range(n_v * (n_v - 1) // 2))
    tidx = [oracle.triple_index(i, j, k, n_v) for j in range(n_v) for i in range(j)
            for k in range(j + 1, n_v)]
    assert tidx == list(range(n_v * (n_v - 1) * (n_v - 2) // 6))


def test_sampled_rows_and_pairs_agree_with_full():
    geno = synth.panel_hwe(30, 257, seed=9, pad_seed=1)
    full_t, full_c = oracle.ccc2_all(geno, 257)
    rows = np.array([17, 2, 29, 0])
    t, c = oracle.ccc2_rows(geno, 257, rows)
    o = 0
    for i in rows:
        for j in range(i + 1, 30):
            np.testing.assert_array_equal(t[o], full_t[oracle.pair_index(i, j, 30)])
            o += 1
    pi = np.array([0, 5, 28])
    pj = np.array([1, 20, 29])
    t2, c2 = oracle.ccc2_pairs(geno, 257, pi, pj)
    np.testing.assert_array_equal(t2, full_t[oracle.pair_index(pi, pj, 30)])
    np.testing.assert_array_equal(c2, full_c[oracle.pair_index(pi, pj, 30)])
    f3t, f3c = oracle.ccc3_slabs(np.ascontiguousarray(geno[:12]), 257)
    t3, c3 = oracle.ccc3_triples(np.ascontiguousarray(geno[:12]), 257, [0, 3], [4, 5], [11, 6])
    np.testing.assert_array_equal(t3, f3t[oracle.triple_index(np.array([0, 3]), np.array([4, 5]),
                                                              np.array([11, 6]), 12)])
    part_t, _ = oracle.ccc3_slabs(np.ascontiguousarray(geno[:12]), 257, 4, 7)
    lo = oracle.slab_offset(4, 12)
    hi = oracle.slab_offset(7, 12)
    np.testing.assert_array_equal(part_t, f3t[lo:hi])


def test_padding_bits_ignored():
    codes = np.random.default_rng(0).integers(0, 4, size=(6, 45), dtype=np.uint8)
    clean = synth.pack(codes, ld=4)
    dirty = synth.pack(codes, ld=4, pad_seed=77)
    assert np.any(clean != dirty)
    a, ca = oracle.ccc2_all(clean, 45)
    b, cb = oracle.ccc2_all(dirty, 45)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ca, cb)


# ---------------------------------------------------------------- result checksum

def _splitmix_finaliser(x):
    m = (1 << 64) - 1
    z = ((x + 1) * 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def test_checksum_against_big_integer_arithmetic():
    rng = np.random.default_rng(5)
    for n, base in ((1, 0), (1000, 0), (777, 123456789), (5000, (1 << 40) + 3)):
        v = rng.integers(0, 1 << 31, size=n, dtype=np.int64)
        want = sum(_splitmix_finaliser(base + e) * int(x) for e, x in enumerate(v)) % (1 << 128)
        assert oracle.checksum(v, base) == want
    # float32 words: the bit patterns
    f = rng.random(300).astype(np.float32)
    bits = f.view(np.uint32).astype(np.int64)
    want = sum(_splitmix_finaliser(7 + e) * int(x) for e, x in enumerate(bits)) % (1 << 128)
    assert oracle.checksum(f, 7) == want


def test_checksum_is_additive_over_pieces():
    rng = np.random.default_rng(6)
    v = rng.integers(0, 1 << 24, size=10000, dtype=np.int64)
    whole = oracle.checksum(v)
    parts = sum(oracle.checksum(v[a:b], a) for a, b in ((0, 17), (17, 5000), (5000, 10000)))
    assert parts % (1 << 128) == whole
    v2 = v.copy()
    v2[4321] += 1  # one changed value changes the checksum by h(4321)
    assert (oracle.checksum(v2) - whole) % (1 << 128) == _splitmix_finaliser(4321)
