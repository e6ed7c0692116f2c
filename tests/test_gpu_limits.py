"""The largest accepted vector length, n_f = CCC_MAX_NF = 2,097,151.

Every tally is an integer below 8 n_f (3-way) or 4 n_f (2-way), so at the limit
the largest 3-way tally, 8 n_f = 16,777,208, sits just below 2^24 where the
FP32 accumulation stops being exact.  Panels whose entries are all homozygous
(0,0) reach those maxima in closed form (r^{00} = 4 n_f, r^{000} = 8 n_f); a
random panel is checked against the oracle on every pair and triple.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import (assert_ccc_close, assert_tally_equal, run_2way, run_3way, run_multi)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


def _max_nf():
    import paper_1705_08213_gb300 as ccc
    return ccc.CCC_MAX_NF


def _all_hom0(n_v, n_f):
    return synth.pack(np.zeros((n_v, n_f), np.uint8))  # code 00 everywhere


@pytest.mark.parametrize("path", [0, 1])
def test_2way_at_the_length_limit(path):
    n_f = _max_nf()
    t, c = run_2way(_all_hom0(4, n_f), n_f, path)
    assert np.all(t[:, 0] == 4 * n_f) and np.all(t[:, 1:] == 0)
    # every CCC(0,0) = 1 * (1 - 2/3)^2
    np.testing.assert_allclose(c[:, 0], 1.0 / 9.0, rtol=1e-6)
    geno = synth.panel_hwe(5, n_f, seed=61, p_missing=0.01)
    t, c = run_2way(geno, n_f, path)
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t, et, "n_f limit")
    assert_ccc_close(c, ec, what="n_f limit")


@pytest.mark.parametrize("tile", [1, 2])
def test_2way_unsplit_accumulator_at_the_length_limit(tile):
    # With the K split off, one FP32 accumulator per tally sums all n_f individuals:
    # r^{00} of an all-(0,0) pair reaches 4 n_f = 8,388,604 in a single accumulator.
    n_f = _max_nf()
    t, c = run_2way(_all_hom0(4, n_f), n_f, 0, tile=tile, split=1)
    assert np.all(t[:, 0] == 4 * n_f) and np.all(t[:, 1:] == 0)
    np.testing.assert_allclose(c[:, 0], 1.0 / 9.0, rtol=1e-6)
    geno = synth.panel_hwe(5, n_f, seed=63, p_missing=0.01)
    t, c = run_2way(geno, n_f, 0, tile=tile, split=1)
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t, et, "unsplit at the n_f limit")
    assert_ccc_close(c, ec, what="unsplit at the n_f limit")


@pytest.mark.parametrize("path,tile", [(0, 0), (0, 1), (1, 0)])
def test_3way_at_the_length_limit(path, tile):
    n_f = _max_nf()
    t, c = run_3way(_all_hom0(4, n_f), n_f, path, tile=tile)
    assert np.all(t[:, 0] == 8 * n_f) and np.all(t[:, 1:] == 0)
    assert 8 * n_f < 1 << 24
    geno = synth.panel_hwe(5, n_f, seed=62, p_missing=0.01)
    t, c = run_3way(geno, n_f, path, tile=tile)
    et, ec = oracle.ccc3_slabs(geno, n_f)
    assert_tally_equal(t, et, "n_f limit")
    assert_ccc_close(c, ec, what="n_f limit")


def test_multi_at_the_length_limit():
    n_f = _max_nf()
    g = np.zeros((3, synth.multi_default_ld(n_f)), np.uint8)  # state (0, 0) everywhere
    t, c = run_multi(g, n_f, 2)
    assert np.all(t[:, 0] == 4 * n_f) and np.all(t[:, 1:] == 0)
