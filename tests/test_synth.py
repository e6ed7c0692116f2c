"""Input generators and the packed 2-bit storage format (host only)."""

import numpy as np
import pytest

import synth


def test_pack_unpack_roundtrip_all_tails():
    rng = np.random.default_rng(5)
    for n_f in (1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 1000):
        codes = rng.integers(0, 4, size=(7, n_f), dtype=np.uint8)
        for pad_seed in (None, 3):
            w = synth.pack(codes, pad_seed=pad_seed)
            assert w.shape == (7, synth.default_ld(n_f))
            assert synth.default_ld(n_f) % 2 == 0
            np.testing.assert_array_equal(synth.unpack(w, n_f), codes)


def test_pack_bit_positions():
    # entry q sits at bits 2*(q%32) of word q//32, LSB first
    codes = np.zeros((1, 70), np.uint8)
    codes[0, 0] = 0b11
    codes[0, 33] = 0b10
    codes[0, 69] = 0b01
    w = synth.pack(codes, ld=4)
    assert int(w[0, 0]) == 0b11
    assert int(w[0, 1]) == 0b10 << 2
    assert int(w[0, 2]) == 0b01 << (2 * 5)
    assert int(w[0, 3]) == 0


def test_padding_garbage_is_nonzero_and_outside_entries():
    codes = np.zeros((4, 40), np.uint8)
    w = synth.pack(codes, ld=6, pad_seed=11)
    # entries 0..39 are zero; the remaining bits of word 1 and words 2..5 hold garbage
    assert np.all(w[:, 0] == 0)
    assert np.all(w[:, 1] & np.uint64((1 << 16) - 1) == 0)
    assert np.any(w[:, 1] >> np.uint64(16) != 0)
    assert np.any(w[:, 2:] != 0)


def test_genotype_codes():
    g = np.array([[0, 1, 2, -1]])
    np.testing.assert_array_equal(synth.codes_from_genotypes(g), [[0b00, 0b01, 0b11, 0b10]])


def test_generators_deterministic_and_counter_based():
    a = synth.panel_hwe(50, 300, seed=7)
    b = synth.panel_hwe(50, 300, seed=7)
    np.testing.assert_array_equal(a, b)
    # any row can be regenerated on its own
    g_rows = synth.genotypes_hwe(7, 0, np.array([13, 41]), 300, 0.01)
    codes = synth.unpack(a, 300)
    np.testing.assert_array_equal(synth.codes_from_genotypes(g_rows), codes[[13, 41]])
    c = synth.panel_hwe(50, 300, seed=8)
    assert np.any(a != c)


def test_uniform_panel_statistics():
    g = synth.genotypes_uniform(0, 0, np.arange(256), 1024, 0.02)
    miss = np.mean(g < 0)
    assert abs(miss - 0.02) < 0.003
    present = g[g >= 0]
    for v in (0, 1, 2):
        assert abs(np.mean(present == v) - 1 / 3) < 0.01


def test_hwe_panel_statistics():
    snps = np.arange(400)
    p = synth.maf_beta_half(1, 0, snps)
    assert p.min() >= 0.01 and p.max() <= 0.5
    g = synth.genotypes_hwe(1, 0, snps, 4000, 0.01)
    assert abs(np.mean(g < 0) - 0.01) < 0.002
    # per-SNP allele frequency of the drawn genotypes tracks p
    gg = np.where(g < 0, np.nan, g.astype(float))
    phat = np.nanmean(gg, axis=1) / 2
    assert np.max(np.abs(phat - p)) < 0.05
    # Hardy-Weinberg: heterozygote share ~ 2p(1-p)
    het = np.nanmean(np.where(np.isnan(gg), np.nan, gg == 1), axis=1)
    assert np.mean(np.abs(het - 2 * p * (1 - p))) < 0.02


def test_beta_half_folded_distribution():
    # Beta(1/2,1/2) folded to [0,1/2]: P(p <= t) = (4/pi) asin(sqrt(t)) for t in [0, 1/2]
    p = synth.maf_beta_half(3, 0, np.arange(200000))
    for t in (0.05, 0.1, 0.25, 0.4):
        expect = 4 / np.pi * np.arcsin(np.sqrt(t))
        assert abs(np.mean(p <= t) - expect) < 0.005


def test_ld_too_small_rejected():
    with pytest.raises(ValueError):
        synth.pack(np.zeros((1, 65), np.uint8), ld=2)


@pytest.mark.parametrize("n_f", [1, 31, 32, 33, 100, 1000])
def test_fast_generator_equals_numpy_definition(n_f):
    """The C twin of the generator reproduces the numpy definitions bit for bit."""
    assert synth._fast_lib() is not None
    for fn, kw in ((synth.panel_uniform, dict(seed=0, p_missing=0.02)),
                   (synth.panel_hwe, dict(seed=4, p_missing=0.05))):
        for pad in (None, 5):
            a = fn(37, n_f, pad_seed=pad, fast=True, **kw)
            b = fn(37, n_f, pad_seed=pad, fast=False, **kw)
            np.testing.assert_array_equal(a, b)
