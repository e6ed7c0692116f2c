"""K-split 2-way calls (ccc_opts.split): panels with few SNP tiles and long vectors.

The individuals are split into parts whose partial tallies are summed on the
device (the n_pf axis of Sec. 4 on one GPU); CCC values then come from the
summed tallies.  Results must equal the unsplit call bit for bit and the
oracle exactly (tallies) / within 1e-6 (CCC), for forced and automatic splits,
both normalisations, tally-only calls, and outputs in pinned host memory
(which the split does not use); on the tensor cores (biallelic and s-state) and
on the popcount path.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_ccc_close, assert_tally_equal, to_device, workspace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


def _run(geno, n_f, split, norm=0, tally_only=False, host=False, operand=0):
    import torch

    import paper_1705_08213_gb300 as ccc
    g = to_device(geno)
    n_v = geno.shape[0]
    opts = ccc.ccc_opts_default(norm=norm)
    opts.operand = operand
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(norm=norm, workspace=ws)
    opts.split = split
    opts.operand = operand
    npairs = ccc.ccc2_count(n_v)
    kw = dict(dtype=torch.int32, pin_memory=True) if host else dict(dtype=torch.int32, device="cuda")
    tally = torch.full((npairs, 4), -7, **kw)
    kwf = dict(kw, dtype=torch.float32)
    out = torch.full((npairs, 4), -7.0, **kwf)
    if tally_only:
        ccc.ccc2_tally(g, n_f, tally, opts)
    else:
        ccc.ccc2_tally_metric(g, n_f, tally, out, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    return tally.cpu().numpy(), out.cpu().numpy()


@pytest.mark.parametrize("operand", [0, 1])  # automatic (e2m1), e4m3
@pytest.mark.parametrize("norm", [0, 1])
def test_forced_splits_equal_unsplit_and_oracle(norm, operand):
    # 300 SNPs: not a multiple of the unpack's 32-SNP blocks; 5,000 individuals:
    # a ragged last K block (20 e2m1 / 40 e4m3 K stages).
    n_v, n_f = 300, 5000
    geno = synth.panel_hwe(n_v, n_f, seed=71, p_missing=0.02)
    t1, c1 = _run(geno, n_f, 1, norm, operand=operand)
    et, ec = oracle.ccc2_all(geno, n_f, norm=norm)
    assert_tally_equal(t1, et, "unsplit")
    assert_ccc_close(c1, ec, what="unsplit")
    for split in (2, 3, 7, 40, 4096):  # 4096 is clamped to the K stages
        t, c = _run(geno, n_f, split, norm, operand=operand)
        np.testing.assert_array_equal(t, t1)
        np.testing.assert_array_equal(c, c1)


def test_automatic_split_on_a_long_panel():
    n_v, n_f = 500, 100000
    geno = synth.panel_hwe(n_v, n_f, seed=72, p_missing=0.01)
    t, c = _run(geno, n_f, 0)
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t, et, "auto split")
    assert_ccc_close(c, ec, what="auto split")
    t1, c1 = _run(geno, n_f, 1)
    np.testing.assert_array_equal(t, t1)
    np.testing.assert_array_equal(c, c1)


@pytest.mark.parametrize("operand", [0, 1])  # automatic (e2m1), e4m3
def test_forced_split_many_snps(operand):
    """1,300 SNPs (1,536 padded): the K-block-major unpack runs 48 blocks of 32
    SNPs over several K ranges each, the per-SNP counts summed by atomics
    across the ranges; 3,000 individuals end in a ragged K block."""
    n_v, n_f = 1300, 3000
    geno = synth.panel_hwe(n_v, n_f, seed=76, p_missing=0.03)
    t1, c1 = _run(geno, n_f, 1, operand=operand)
    t3, c3 = _run(geno, n_f, 3, operand=operand)
    np.testing.assert_array_equal(t3, t1)
    np.testing.assert_array_equal(c3, c1)
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t3, et, "split 3")
    assert_ccc_close(c3, ec, what="split 3")


@pytest.mark.parametrize("operand", [0, 1])  # automatic (e2m1), e4m3
@pytest.mark.parametrize("n_v, n_f", [(2, 511), (3, 512), (40, 513), (33, 8191), (65, 8192)])
def test_forced_split_at_k_block_edges(n_v, n_f, operand):
    """n_f at and around a 128-byte K block (256 e2m1 / 128 e4m3 entries), few SNPs: the
    K-block-major unpack's last block and its per-SNP counts, split 2 against unsplit."""
    geno = synth.panel_hwe(n_v, n_f, seed=78 + n_v, p_missing=0.05)
    t1, c1 = _run(geno, n_f, 1, operand=operand)
    t2, c2 = _run(geno, n_f, 2, operand=operand)
    np.testing.assert_array_equal(t2, t1)
    np.testing.assert_array_equal(c2, c1)
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t2, et, "split 2")
    assert_ccc_close(c2, ec, what="split 2")


def test_tally_only_and_host_outputs():
    n_v, n_f = 200, 9000
    geno = synth.panel_hwe(n_v, n_f, seed=73, p_missing=0.02)
    et, ec = oracle.ccc2_all(geno, n_f)
    t, _ = _run(geno, n_f, 5, tally_only=True)
    assert_tally_equal(t, et, "tally only")
    t, c = _run(geno, n_f, 5, host=True)  # pinned host outputs: computed unsplit
    assert_tally_equal(t, et, "host outputs")
    assert_ccc_close(c, ec, what="host outputs")


@pytest.mark.parametrize("s", [3, 4, 11])
def test_multi_split_equals_unsplit_and_oracle(s):
    import torch

    import paper_1705_08213_gb300 as ccc
    from tests.gpu_util import to_device_bytes
    n_v, n_f = 90, 20000
    gm = synth.panel_multi(n_v, n_f, s, seed=75 + s, p_missing=0.02)
    g = to_device_bytes(gm)
    res = {}
    for split in (1, 0, 6):
        opts = ccc.ccc_opts_default()
        ws = workspace(ccc.ccc_multi_workspace_size(g, n_f, s, opts))
        opts = ccc.ccc_opts_default(workspace=ws)
        opts.split = split
        npairs = ccc.ccc2_count(n_v)
        t = torch.full((npairs, s * s), -7, dtype=torch.int32, device="cuda")
        c = torch.full((npairs, s * s), -7.0, dtype=torch.float32, device="cuda")
        ccc.ccc2_multi_tally_metric(g, n_f, s, t, c, opts)
        torch.cuda.synchronize()
        assert ccc.ccc_status(opts) == ccc.CCC_OK
        res[split] = (t.cpu().numpy(), c.cpu().numpy())
    et, ec = oracle.ccc2_multi_all(gm, n_f, s)
    assert_tally_equal(res[1][0], et, "multi unsplit")
    assert_ccc_close(res[1][1], ec, what="multi unsplit")
    for split in (0, 6):
        np.testing.assert_array_equal(res[split][0], res[1][0])
        np.testing.assert_array_equal(res[split][1], res[1][1])



def _run_path(geno, n_f, split, path, norm=0):
    import torch

    import paper_1705_08213_gb300 as ccc
    g = to_device(geno)
    n_v = geno.shape[0]
    opts = ccc.ccc_opts_default(path=path, norm=norm)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(path=path, norm=norm, workspace=ws)
    opts.split = split
    npairs = ccc.ccc2_count(n_v)
    tally = torch.full((npairs, 4), -7, dtype=torch.int32, device="cuda")
    out = torch.full((npairs, 4), -7.0, dtype=torch.float32, device="cuda")
    ccc.ccc2_tally_metric(g, n_f, tally, out, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    return tally.cpu().numpy(), out.cpu().numpy()


@pytest.mark.parametrize("norm", [0, 1])
def test_popc_forced_splits_equal_unsplit_and_oracle(norm):
    """The popcount path's K split: parts of whole 8-word stages whose partial tallies are
    summed with integer reductions, CCC values from the sums."""
    n_v, n_f = 150, 9000 + 37  # 18 stages of 512 individuals, ragged
    geno = synth.panel_hwe(n_v, n_f, seed=76, p_missing=0.02, pad_seed=3)
    et, ec = oracle.ccc2_all(geno, n_f, norm=norm)
    t1, c1 = _run_path(geno, n_f, 1, 1, norm)
    assert_tally_equal(t1, et, "popc unsplit")
    assert_ccc_close(c1, ec, what="popc unsplit")
    for split in (2, 5, 18, 4096):  # 4096 is clamped to the 18 stages
        t, c = _run_path(geno, n_f, split, 1, norm)
        np.testing.assert_array_equal(t, t1)
        np.testing.assert_array_equal(c, c1)


def test_popc_automatic_split_on_a_long_panel():
    n_v, n_f = 300, 200000 + 5
    geno = synth.panel_hwe(n_v, n_f, seed=77, p_missing=0.01, pad_seed=4)
    t, c = _run_path(geno, n_f, 0, 1)
    t_tc, c_tc = _run_path(geno, n_f, 0, 0)
    np.testing.assert_array_equal(t, t_tc)
    np.testing.assert_array_equal(c, c_tc)
    rows = np.array([0, 150, 298])
    et, ec = oracle.ccc2_rows(geno, n_f, rows)
    idx = np.concatenate([oracle.pair_index(i, np.arange(i + 1, n_v), n_v) for i in rows])
    assert_tally_equal(t[idx], et, "popc auto split rows")
    assert_ccc_close(c[idx], ec, what="popc auto split rows")
