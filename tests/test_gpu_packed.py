"""GPU parity of the 2-way pair kernels that expand the 2-bit codes in shared memory
(ccc_opts.tile = 3): the tally kernel reads the packed panel with TMA, and converter warps
write the e4m3 count rows (Sec. 2.1) into the swizzled operand stages; no operand matrix
exists in HBM.

* Against the oracle on panels spanning several 128-SNP tiles with ragged n_v and n_f
  (not multiples of 16, 32 or 128 entries) and garbage in the padding bits past n_f and
  in the padding words of each row, both normalisations.
* Bit for bit against the operand-matrix pair kernel (tile 2): tallies and CCC values,
  row ranges (phases), the streamed output, the thresholded output and K splits.
* The longest accepted vectors (n_f = 2,097,151).
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_ccc_close, assert_tally_equal, run_2way, to_device, workspace

pytestmark = pytest.mark.gpu

PACKED = 3
PAIR = 2


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


@pytest.mark.parametrize("n_v,n_f", [(2, 1), (3, 17), (64, 129), (65, 15), (127, 1000),
                                     (128, 128), (129, 257), (255, 4129), (300, 777),
                                     (600, 3001)])
@pytest.mark.parametrize("norm", [0, 1])
def test_packed_against_oracle(n_v, n_f, norm):
    geno = synth.panel_uniform(n_v, n_f, seed=900 + n_v, p_missing=0.03, pad_seed=n_v + 1)
    t, c = run_2way(geno, n_f, 0, norm=norm, tile=PACKED)
    et, ec = oracle.ccc2_all(geno, n_f, norm=norm)
    assert_tally_equal(t, et, f"packed n_v={n_v} n_f={n_f}")
    assert_ccc_close(c, ec, what=f"packed n_v={n_v} n_f={n_f}")


@pytest.mark.parametrize("n_v,n_f,ld", [(1000, 20000, None), (1500, 6000, 200), (333, 1000, 40)])
def test_packed_equals_operand_matrix(n_v, n_f, ld):
    geno = synth.panel_hwe(n_v, n_f, seed=n_v, p_missing=0.01, ld=ld, pad_seed=7)
    for norm in (0, 1):
        t2, c2 = run_2way(geno, n_f, 0, norm=norm, tile=PAIR)
        t3, c3 = run_2way(geno, n_f, 0, norm=norm, tile=PACKED)
        np.testing.assert_array_equal(t3, t2)
        np.testing.assert_array_equal(c3, c2)
    rows = np.array([0, n_v // 2, n_v - 2])
    et, _ = oracle.ccc2_rows(geno, n_f, rows)
    idx = np.concatenate([oracle.pair_index(i, np.arange(i + 1, n_v), n_v) for i in rows])
    assert_tally_equal(t3[idx], et, "packed rows")


def test_packed_tally_only_and_separate_metric():
    n_v, n_f = 400, 2500
    geno = synth.panel_hwe(n_v, n_f, seed=91, p_missing=0.02, pad_seed=3)
    t, c = run_2way(geno, n_f, 0, tile=PACKED, fused=False)
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t, et, "packed tally only")
    assert_ccc_close(c, ec, what="packed, metric from stored tallies")


def test_packed_row_ranges_and_stream():
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 700, 2000
    geno = synth.panel_hwe(n_v, n_f, seed=92, p_missing=0.01, pad_seed=4)
    full_t, full_c = run_2way(geno, n_f, 0, tile=PAIR)
    g = to_device(geno)
    opts = ccc.ccc_opts_default(tile=PACKED)
    ws = workspace(ccc.ccc2_stream_workspace_size(g, n_f, 5, opts))
    opts = ccc.ccc_opts_default(workspace=ws, tile=PACKED)
    for i0, i1 in ((0, 128), (100, 400), (640, 700)):
        cnt = ccc.ccc2_rows_count(n_v, i0, i1)
        t = torch.empty((cnt, 4), dtype=torch.int32, device="cuda")
        c = torch.empty((cnt, 4), dtype=torch.float32, device="cuda")
        ccc.ccc2_tally_metric_rows(g, n_f, i0, i1, t, c, opts)
        torch.cuda.synchronize()
        assert ccc.ccc_status(opts) == ccc.CCC_OK
        p0 = ccc.ccc2_index(i0, i0 + 1, n_v)
        np.testing.assert_array_equal(t.cpu().numpy(), full_t[p0:p0 + cnt])
        np.testing.assert_array_equal(c.cpu().numpy(), full_c[p0:p0 + cnt])
    npairs = ccc.ccc2_count(n_v)
    ht = torch.full((npairs, 4), -7, dtype=torch.int32, pin_memory=True)
    hc = torch.full((npairs, 4), -7.0, dtype=torch.float32, pin_memory=True)
    ccc.ccc2_stream(g, n_f, 5, ht, hc, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    np.testing.assert_array_equal(ht.numpy(), full_t)
    np.testing.assert_array_equal(hc.numpy(), full_c)


def _filter(geno, n_f, tile, threshold, cap):
    import torch

    import paper_1705_08213_gb300 as ccc
    g = to_device(geno)
    opts = ccc.ccc_opts_default(tile=tile)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(tile=tile, workspace=ws)
    hits = torch.zeros(cap * 40, dtype=torch.uint8, device="cuda")
    n_hits = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    ccc.ccc2_filter(g, n_f, threshold, hits, cap, n_hits, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    total = int(n_hits.item())
    rec = hits.cpu().numpy().reshape(cap, 40)[:min(total, cap)]
    order = np.lexsort((rec[:, 4:8].view(np.int32)[:, 0], rec[:, 0:4].view(np.int32)[:, 0]))
    return total, rec[order]


def test_packed_thresholded_output_equals_operand_matrix():
    n_v, n_f, tau = 600, 1000, 0.155
    geno = synth.panel_hwe(n_v, n_f, seed=93, p_missing=0.01, pad_seed=2)
    synth.plant_near_duplicates(geno, n_f, 60, seed=19)
    total2, rec2 = _filter(geno, n_f, PAIR, tau, 10000)
    total3, rec3 = _filter(geno, n_f, PACKED, tau, 10000)
    assert total2 >= 10 and total3 == total2
    np.testing.assert_array_equal(rec3, rec2)


def _split_run(geno, n_f, tile, split):
    import torch

    import paper_1705_08213_gb300 as ccc
    g = to_device(geno)
    n_v = geno.shape[0]
    opts = ccc.ccc_opts_default(tile=tile)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(tile=tile, workspace=ws)
    opts.split = split
    npairs = ccc.ccc2_count(n_v)
    t = torch.full((npairs, 4), -7, dtype=torch.int32, device="cuda")
    c = torch.full((npairs, 4), -7.0, dtype=torch.float32, device="cuda")
    ccc.ccc2_tally_metric(g, n_f, t, c, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    return t.cpu().numpy(), c.cpu().numpy()


def test_packed_k_split():
    n_v, n_f = 300, 5000 + 77  # 40 K stages, ragged
    geno = synth.panel_hwe(n_v, n_f, seed=94, p_missing=0.02, pad_seed=5)
    et, ec = oracle.ccc2_all(geno, n_f)
    t1, c1 = _split_run(geno, n_f, PACKED, 1)
    assert_tally_equal(t1, et, "packed unsplit")
    assert_ccc_close(c1, ec, what="packed unsplit")
    for split in (2, 7, 40, 4096):
        t, c = _split_run(geno, n_f, PACKED, split)
        np.testing.assert_array_equal(t, t1)
        np.testing.assert_array_equal(c, c1)


def test_packed_automatic_split_on_a_long_panel():
    n_v, n_f = 500, 100000 + 3
    geno = synth.panel_hwe(n_v, n_f, seed=95, p_missing=0.01, pad_seed=6)
    t, c = _split_run(geno, n_f, PACKED, 0)
    t2, c2 = _split_run(geno, n_f, PAIR, 0)
    np.testing.assert_array_equal(t, t2)
    np.testing.assert_array_equal(c, c2)
    rows = np.array([0, 255, 498])
    et, ec = oracle.ccc2_rows(geno, n_f, rows)
    idx = np.concatenate([oracle.pair_index(i, np.arange(i + 1, n_v), n_v) for i in rows])
    assert_tally_equal(t[idx], et, "packed long rows")
    assert_ccc_close(c[idx], ec, what="packed long rows")


def test_packed_at_the_length_limit():
    import paper_1705_08213_gb300 as ccc
    n_f = ccc.CCC_MAX_NF
    t, c = run_2way(synth.pack(np.zeros((4, n_f), np.uint8)), n_f, 0, tile=PACKED)
    assert np.all(t[:, 0] == 4 * n_f) and np.all(t[:, 1:] == 0)
    geno = synth.panel_hwe(5, n_f, seed=96, p_missing=0.01, pad_seed=8)
    t, c = run_2way(geno, n_f, 0, tile=PACKED)
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t, et, "packed n_f limit")
    assert_ccc_close(c, ec, what="packed n_f limit")


def test_packed_degenerate_snps():
    """An all-missing SNP, identical SNPs and a half-missing SNP (codes built on the host)."""
    n_v, n_f = 70, 300
    codes = synth.unpack(synth.panel_hwe(n_v, n_f, seed=97, p_missing=0.02), n_f)
    codes[5] = 2          # all missing
    codes[7] = codes[8]   # identical
    codes[11, :100] = 2   # first 100 entries missing
    geno = synth.pack(codes, pad_seed=9)
    for norm in (0, 1):
        t, c = run_2way(geno, n_f, 0, norm=norm, tile=PACKED)
        et, ec = oracle.ccc2_all(geno, n_f, norm=norm)
        assert_tally_equal(t, et, "packed degenerate SNPs")
        assert_ccc_close(c, ec, what="packed degenerate SNPs")
