"""GPU parity of the 2-way path (tensor-core and popcount) against the CPU oracle.

Tallies must match bit for bit; CCC values within 1e-6 relative (the bound of
the single-precision epilogue, derived in csrc/ccc_metric.cuh).
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_ccc_close, assert_tally_equal, run_2way

pytestmark = pytest.mark.gpu

PATHS = [0, 1]  # CCC_PATH_TC, CCC_PATH_POPC
NF_EDGES = [1, 31, 32, 33, 63, 64, 65, 127, 128, 129, 1000]
NV_EDGES = [2, 3, 4, 63, 64, 65, 129, 300]


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


def _check(geno, n_f, path, norm=0, gamma=2.0 / 3.0, fused=True):
    t, c = run_2way(geno, n_f, path, norm=norm, gamma=gamma, fused=fused)
    et, ec = oracle.ccc2_all(geno, n_f, gamma=gamma, norm=norm)
    assert_tally_equal(t, et, f"tally n_v={geno.shape[0]} n_f={n_f} path={path}")
    assert_ccc_close(c, ec, what=f"ccc n_v={geno.shape[0]} n_f={n_f} path={path} norm={norm}")


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n_f", NF_EDGES)
@pytest.mark.parametrize("n_v", [2, 65, 129])
def test_shapes_nf_edges(path, n_f, n_v):
    geno = synth.panel_uniform(n_v, n_f, seed=100 + n_f, p_missing=0.05, pad_seed=n_f + 3)
    _check(geno, n_f, path)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n_v", NV_EDGES)
@pytest.mark.parametrize("n_f", [1, 129, 1000])
def test_shapes_nv_edges(path, n_v, n_f):
    geno = synth.panel_hwe(n_v, n_f, seed=200 + n_v, p_missing=0.02, pad_seed=n_v)
    _check(geno, n_f, path)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("norm", [0, 1])
def test_small_uniform_panel(path, norm):
    """256 SNPs x 1024 individuals, uniform genotypes, 2% missing, seed 0."""
    geno = synth.panel_uniform(256, 1024, seed=0, p_missing=0.02)
    _check(geno, 1024, path, norm=norm)
    _check(geno, 1024, path, norm=norm, fused=False)


@pytest.mark.parametrize("path", PATHS)
def test_gamma_values(path):
    geno = synth.panel_hwe(70, 300, seed=5, p_missing=0.03)
    for gamma in (0.0, 0.25, 1.0):
        _check(geno, 300, path, gamma=gamma)


@pytest.mark.parametrize("path", PATHS)
def test_degenerate_snps(path):
    n_f = 200
    g = synth.genotypes_uniform(3, 0, np.arange(40), n_f, 0.05)
    g[5] = -1           # an all-missing SNP
    g[7] = g[8]         # identical SNPs
    g[9] = 0            # monomorphic SNP
    g[10] = 2
    g[11, :100] = -1    # half missing
    geno = synth.pack(synth.codes_from_genotypes(g), pad_seed=1)
    _check(geno, n_f, path)
    _check(geno, n_f, path, norm=1)


@pytest.mark.parametrize("path", PATHS)
def test_wide_row_stride(path):
    codes = synth.codes_from_genotypes(synth.genotypes_hwe(4, 0, np.arange(90), 130, 0.01))
    geno = synth.pack(codes, ld=12, pad_seed=9)  # ld well above ceil(130/32) = 5
    _check(geno, 130, path)


def test_single_snp_has_no_pairs():
    geno = synth.panel_uniform(1, 50, seed=1)
    for path in PATHS:
        t, c = run_2way(geno, 50, path)
        assert t.shape == (0, 4) and c.shape == (0, 4)


def test_allele_counts():
    import torch

    import paper_1705_08213_gb300 as ccc
    from tests.gpu_util import to_device
    for n_v, n_f in ((1, 1), (37, 33), (300, 1000), (129, 4097)):
        geno = synth.panel_hwe(n_v, n_f, seed=n_f, p_missing=0.05, pad_seed=2)
        counts = torch.zeros((n_v, 3), dtype=torch.int32, device="cuda")
        ccc.ccc_allele_counts(to_device(geno), n_f, counts)
        s0, s1, npres = oracle.allele_counts(geno, n_f)
        np.testing.assert_array_equal(counts.cpu().numpy(), np.stack([s0, s1, npres], 1))


def test_at_scale_tc_equals_popc_and_oracle_rows():
    """20,000 SNPs x 16,384 individuals (Hardy-Weinberg, Beta(1/2,1/2) MAF, 1% missing):
    the tensor-core tallies, with FP4 (the automatic operands) and with e4m3 operands,
    equal the popcount tallies on every pair (tallies reach 4 n_f = 65,536, far past the
    exact range of narrower accumulators), and sampled rows equal the oracle."""
    import torch

    import paper_1705_08213_gb300 as ccc
    from tests.gpu_util import to_device, workspace
    n_v, n_f = 20000, 16384
    geno = synth.panel_hwe(n_v, n_f, seed=1, p_missing=0.01)
    g = to_device(geno)
    npairs = ccc.ccc2_count(n_v)
    outs = {}
    for path in PATHS + ["e4m3"]:
        operand = ccc.CCC_OPERAND_E4M3 if path == "e4m3" else ccc.CCC_OPERAND_AUTO
        path_id = 0 if path == "e4m3" else path
        opts = ccc.ccc_opts_default(path=path_id, operand=operand)
        ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
        opts = ccc.ccc_opts_default(path=path_id, workspace=ws, operand=operand)
        tally = torch.empty((npairs, 4), dtype=torch.int32, device="cuda")
        out = torch.empty((npairs, 4), dtype=torch.float32, device="cuda")
        ccc.ccc2_tally_metric(g, n_f, tally, out, opts)
        torch.cuda.synchronize()
        assert ccc.ccc_status(opts) == ccc.CCC_OK
        outs[path] = (tally, out)
        del ws
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])
    assert torch.equal(outs[0][0], outs["e4m3"][0])
    assert torch.equal(outs[0][1], outs["e4m3"][1])
    # row sums of each table are 4 n_ij <= 4 n_f
    s = outs[0][0].sum(dim=1, dtype=torch.int64)
    assert int(s.max()) <= 4 * n_f and int(s.min()) >= 0
    rows = np.array([0, 1, 63, 64, 127, 128, 9999, 17011, n_v - 2])
    et, ec = oracle.ccc2_rows(geno, n_f, rows)
    idx = np.concatenate([oracle.pair_index(i, np.arange(i + 1, n_v), n_v) for i in rows])
    idx_t = torch.from_numpy(idx).cuda()
    assert_tally_equal(outs[0][0][idx_t].cpu().numpy(), et, "sampled rows")
    assert_ccc_close(outs[0][1][idx_t].cpu().numpy(), ec, what="sampled rows")
