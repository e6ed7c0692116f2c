"""GPU parity of the 3-way path (tensor-core and popcount) against the CPU oracle.

Tallies bit for bit; CCC values within 1e-6 relative.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_ccc_close, assert_tally_equal, run_3way

pytestmark = pytest.mark.gpu

# (path, tile): tensor cores by genotype classes of v_j on SM pairs (default), tensor cores
# with the masked operand L_j formed in HBM first, L_j formed in shared memory, popcount.
PATHS = [(0, 0), (0, 1), (0, 2), (1, 0)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


def _check(geno, n_f, path, j_begin=0, j_end=None, norm=0, gamma=2.0 / 3.0, fused=True):
    n_v = geno.shape[0]
    j_end = n_v if j_end is None else j_end
    path, tile = path
    t, c = run_3way(geno, n_f, path, j_begin, j_end, norm=norm, gamma=gamma, fused=fused,
                    tile=tile)
    et, ec = oracle.ccc3_slabs(geno, n_f, j_begin, j_end, gamma=gamma, norm=norm)
    what = f"n_v={n_v} n_f={n_f} path={path} j=[{j_begin},{j_end}) norm={norm}"
    assert_tally_equal(t, et, "tally " + what)
    assert_ccc_close(c, ec, what="ccc " + what)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n_v", [3, 4, 5, 33, 34, 65, 130])
@pytest.mark.parametrize("n_f", [1, 33, 129, 300])
def test_shapes(path, n_v, n_f):
    geno = synth.panel_uniform(n_v, n_f, seed=400 + n_v + n_f, p_missing=0.05, pad_seed=n_f)
    _check(geno, n_f, path)


@pytest.mark.parametrize("path", PATHS)
def test_slab_ranges(path):
    geno = synth.panel_hwe(70, 200, seed=8, p_missing=0.02, pad_seed=2)
    for jb, je in ((0, 1), (5, 9), (33, 34), (60, 70), (69, 70), (0, 70), (40, 40)):
        _check(geno, 200, path, jb, je)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("norm", [0, 1])
def test_norms_and_split_calls(path, norm):
    geno = synth.panel_hwe(50, 257, seed=9, p_missing=0.03)
    _check(geno, 257, path, norm=norm)
    _check(geno, 257, path, 7, 31, norm=norm, fused=False)


@pytest.mark.parametrize("path", PATHS)
def test_gamma_values(path):
    geno = synth.panel_uniform(40, 100, seed=10, p_missing=0.05)
    for gamma in (0.0, 1.0):
        _check(geno, 100, path, gamma=gamma)


@pytest.mark.parametrize("path", PATHS)
def test_degenerate_snps(path):
    n_f = 150
    g = synth.genotypes_uniform(6, 0, np.arange(36), n_f, 0.05)
    g[3] = -1
    g[8] = g[9]
    g[10] = 2
    g[20, :75] = -1
    geno = synth.pack(synth.codes_from_genotypes(g), pad_seed=3)
    _check(geno, n_f, path)
    _check(geno, n_f, path, norm=1)


@pytest.mark.parametrize("path", PATHS)
def test_missing_counts_around_the_compaction_capacity(path):
    """SNPs with exactly 0, 1, 127, 128, 129, 255, 256, 257, 400 and all 600 entries
    missing: the class kernel restricts the missing-column product to 128-column blocks
    of at most 256 individuals and masks all of R beyond that."""
    n_f = 600
    counts = [0, 1, 127, 128, 129, 255, 256, 257, 400, 600]
    g = synth.genotypes_uniform(7, 0, np.arange(3 * len(counts)), n_f, 0.0)
    rng = np.random.default_rng(12)
    for s, m in enumerate(counts):
        g[3 * s, rng.choice(n_f, size=m, replace=False)] = -1
    geno = synth.pack(synth.codes_from_genotypes(g), pad_seed=4)
    _check(geno, n_f, path)
    _check(geno, n_f, path, 5, 21, norm=1)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("p_missing", [0.0, 0.35])
def test_missing_rates(path, p_missing):
    geno = synth.panel_hwe(150, 700, seed=13, p_missing=p_missing, pad_seed=5)
    _check(geno, 700, path)


@pytest.mark.parametrize("path", PATHS)
def test_long_vectors(path):
    """n_f = 16,400 > 16,383: the class route's D counts may pass 16 bits, so it runs the
    narrower tiles that keep D in tensor memory; one SNP has 300 missing entries."""
    n_f = 16400
    geno = synth.panel_hwe(45, n_f, seed=14, p_missing=0.01, pad_seed=6)
    codes = synth.unpack(geno, n_f)
    codes[7, :300] = synth.CODE_MISSING
    geno = synth.pack(codes, pad_seed=6)
    _check(geno, n_f, path)


def test_at_scale_tc_equals_popc_and_oracle_rows():
    """1,536 SNPs x 8,192 individuals (Hardy-Weinberg, 1% missing), all 602,800,640
    triples: the genotype-class tallies (default) equal the popcount tallies and the
    masked-operand tallies (tallies reach 8 n_f = 65,536), CCC values agree, and sampled
    (i, j) rows equal the oracle.  The masked operands of this size span many slab
    batches."""
    import torch

    import paper_1705_08213_gb300 as ccc
    from tests.gpu_util import to_device, workspace
    n_v, n_f = 1536, 8192
    geno = synth.panel_hwe(n_v, n_f, seed=4, p_missing=0.01)
    g = to_device(geno)
    nt = ccc.ccc3_count(n_v, 0, n_v)
    outs = {}
    for path, tile in ((0, 0), (1, 0), (0, 1)):
        opts = ccc.ccc_opts_default(path=path, tile=tile)
        ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_3WAY))
        opts = ccc.ccc_opts_default(path=path, workspace=ws, tile=tile)
        tally = torch.empty((nt, 8), dtype=torch.int32, device="cuda")
        out = torch.empty((nt, 8), dtype=torch.float32, device="cuda")
        ccc.ccc3_tally_metric(g, n_f, 0, n_v, tally, out, opts)
        torch.cuda.synchronize()
        assert ccc.ccc_status(opts) == ccc.CCC_OK
        if tile == 1:  # the masked-operand route must equal the class route
            assert torch.equal(tally, outs[0][0])
            assert torch.equal(out, outs[0][1])
            del tally, out
        else:
            outs[path] = (tally, out)
        del ws
    assert torch.equal(outs[0][0], outs[1][0])
    step = 1 << 25
    for r0 in range(0, nt, step):
        a = outs[0][1][r0:r0 + step].double()
        b = outs[1][1][r0:r0 + step].double()
        assert bool(((a - b).abs() <= 2e-6 * b.abs()).all())
    ri = np.array([0, 5, 700, 31, 1000, 1533])
    rj = np.array([1, 800, 701, 1534, 1400, 1534])
    et, ec = oracle.ccc3_rows(geno, n_f, ri, rj)
    idx = np.concatenate([oracle.triple_index(i, j, np.arange(j + 1, n_v), n_v) for i, j in zip(ri, rj)])
    idx_t = torch.from_numpy(idx).cuda()
    assert_tally_equal(outs[0][0][idx_t].cpu().numpy(), et, "sampled rows")
    assert_ccc_close(outs[0][1][idx_t].cpu().numpy(), ec, what="sampled rows")
