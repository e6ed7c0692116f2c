"""FP4 (e2m1) count operands on the 2-way and 3-way tensor-core paths against the oracle.

Counts 0, 1, 2 are exact in e2m1 (nibbles 0x0, 0x2, 0x4) and every partial sum
is an integer below 2^24, so the block-scaled MMA with unit scale factors must
give tallies bit for bit equal to the oracle's, and CCC values bit for bit equal
to the e4m3 operand path (same tallies, same epilogue).  A 128-byte K stage is
256 entries here, so the n_f edges sit around multiples of 256.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import (assert_ccc_close, assert_tally_equal, run_2way, run_3way, to_device,
                            workspace)

pytestmark = pytest.mark.gpu

E4M3, E2M1 = 1, 2


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


@pytest.mark.parametrize("n_f", [1, 33, 255, 256, 257, 511, 513, 1000, 4097])
@pytest.mark.parametrize("n_v", [2, 129, 300])
def test_fp4_edges_against_oracle(n_v, n_f):
    geno = synth.panel_uniform(n_v, n_f, seed=500 + n_f, p_missing=0.05, pad_seed=n_f + 11)
    t, c = run_2way(geno, n_f, 0, operand=E2M1)
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t, et, f"fp4 tally n_v={n_v} n_f={n_f}")
    assert_ccc_close(c, ec, what=f"fp4 ccc n_v={n_v} n_f={n_f}")


HIT_DTYPE = np.dtype([("i", np.int32), ("j", np.int32), ("tally", np.int32, 4),
                      ("ccc", np.float32, 4)])


# Thresholded FP4 output tiles the triangle by 128 SNPs i x 120 SNPs j (two accumulators of 240
# columns): SNP counts around multiples of 120 and of 128, tile orders of 1 to 64 column blocks,
# both normalisations; a low threshold keeps most pairs, so nearly every tile entry is checked.
@pytest.mark.parametrize("n_v,group,norm", [(119, 0, 0), (120, 0, 1), (121, 0, 0), (240, 0, 0),
                                            (241, 0, 1), (257, 0, 0), (361, 0, 0), (385, 0, 1),
                                            (961, 0, 0), (961, 1, 0), (1500, 3, 1),
                                            (1500, 64, 0)])
def test_fp4_rect_tile_edges(n_v, group, norm):
    import torch

    import paper_1705_08213_gb300 as ccc
    from tests.gpu_util import CCC_RTOL
    n_f, thr = 513, 0.05
    geno = synth.panel_uniform(n_v, n_f, seed=520 + n_v, p_missing=0.05, pad_seed=n_v + 3)
    et, ec = oracle.ccc2_all(geno, n_f, norm=norm)
    g = to_device(geno)
    opts = ccc.ccc_opts_default(norm=norm, operand=E2M1)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(norm=norm, workspace=ws, operand=E2M1)
    opts.group = group
    cap = ccc.ccc2_count(n_v)
    hits = torch.zeros(cap * HIT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n_hits = torch.zeros(1, dtype=torch.int64, device="cuda")
    ccc.ccc2_filter(g, n_f, thr, hits, cap, n_hits, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    n = int(n_hits.item())
    rec = np.frombuffer(hits[:n * HIT_DTYPE.itemsize].cpu().numpy().tobytes(), dtype=HIT_DTYPE)
    ii, jj = np.triu_indices(n_v, 1)
    mx = ec.max(axis=1)
    tie = np.abs(mx - thr) <= CCC_RTOL * thr
    keep = (mx > thr) & ~tie
    assert keep.sum() > 0.5 * keep.size
    got = {(int(h["i"]), int(h["j"])) for h in rec}
    assert len(got) == n
    want = set(zip(ii[keep].tolist(), jj[keep].tolist()))
    assert want <= got <= want | set(zip(ii[tie].tolist(), jj[tie].tolist()))
    idx = oracle.pair_index(rec["i"].astype(np.int64), rec["j"].astype(np.int64), n_v)
    assert_tally_equal(rec["tally"], et[idx], f"fp4 rect tiles n_v={n_v} group={group}")
    assert_ccc_close(rec["ccc"], ec[idx], what=f"fp4 rect tiles n_v={n_v} group={group}")


@pytest.mark.parametrize("norm", [0, 1])
def test_fp4_equals_e4m3_bit_for_bit(norm):
    n_v, n_f = 1100, 5000
    geno = synth.panel_hwe(n_v, n_f, seed=501, p_missing=0.02, pad_seed=12)
    t4, c4 = run_2way(geno, n_f, 0, norm=norm, operand=E2M1)
    t8, c8 = run_2way(geno, n_f, 0, norm=norm, operand=E4M3)
    np.testing.assert_array_equal(t4, t8)
    assert np.array_equal(c4.view(np.int32), c8.view(np.int32)), "CCC bits differ"
    rows = np.array([0, 127, 128, 700, n_v - 2])
    et, ec = oracle.ccc2_rows(geno, n_f, rows, norm=norm)
    idx = np.concatenate([oracle.pair_index(i, np.arange(i + 1, n_v), n_v) for i in rows])
    assert_tally_equal(t4[idx], et, "fp4 sampled rows")
    assert_ccc_close(c4[idx], ec, what="fp4 sampled rows")


def test_fp4_degenerate_snps():
    n_f = 700
    g = synth.genotypes_uniform(3, 0, np.arange(40), n_f, 0.05)
    g[5] = -1           # an all-missing SNP
    g[7] = g[8]         # identical SNPs
    g[9] = 0            # monomorphic SNPs
    g[10] = 2
    g[11, :300] = -1    # half missing
    geno = synth.pack(synth.codes_from_genotypes(g), pad_seed=1)
    for norm in (0, 1):
        t, c = run_2way(geno, n_f, 0, norm=norm, operand=E2M1)
        et, ec = oracle.ccc2_all(geno, n_f, norm=norm)
        assert_tally_equal(t, et, "fp4 degenerate")
        assert_ccc_close(c, ec, what="fp4 degenerate")


@pytest.mark.parametrize("split", [0, 2, 3, 7, 4096])
def test_fp4_k_split(split):
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 300, 40000
    geno = synth.panel_hwe(n_v, n_f, seed=502, p_missing=0.01)
    g = to_device(geno)
    npairs = ccc.ccc2_count(n_v)
    opts = ccc.ccc_opts_default(operand=E2M1)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(workspace=ws, operand=E2M1)
    opts.split = split
    tally = torch.full((npairs, 4), -7, dtype=torch.int32, device="cuda")
    out = torch.full((npairs, 4), -7.0, dtype=torch.float32, device="cuda")
    ccc.ccc2_tally_metric(g, n_f, tally, out, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(tally.cpu().numpy(), et, f"fp4 split={split}")
    assert_ccc_close(out.cpu().numpy(), ec, what=f"fp4 split={split}")


def test_fp4_long_vectors_at_the_length_limit():
    # Unsplit, one FP32 accumulator sums all n_f: r^{00} of all-(0,0) pairs = 4 n_f.
    import paper_1705_08213_gb300 as ccc
    n_f = ccc.CCC_MAX_NF
    geno = synth.pack(np.zeros((4, n_f), np.uint8))
    t, c = run_2way(geno, n_f, 0, split=1, operand=E2M1)
    assert np.all(t[:, 0] == 4 * n_f) and np.all(t[:, 1:] == 0)
    geno = synth.panel_hwe(5, n_f, seed=503, p_missing=0.01)
    for split in (1, 0):
        t, c = run_2way(geno, n_f, 0, split=split, operand=E2M1)
        et, ec = oracle.ccc2_all(geno, n_f)
        assert_tally_equal(t, et, f"fp4 n_f limit split={split}")
        assert_ccc_close(c, ec, what=f"fp4 n_f limit split={split}")


def test_fp4_rows_filter_and_stream():
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 700, 3000
    geno = synth.panel_hwe(n_v, n_f, seed=504, p_missing=0.02)
    synth.plant_near_duplicates(geno, n_f, 30, seed=505)
    g = to_device(geno)
    et, ec = oracle.ccc2_all(geno, n_f)
    opts0 = ccc.ccc_opts_default(operand=E2M1)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts0, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(workspace=ws, operand=E2M1)
    # a row range (one phase)
    lo, hi = 128, 450
    cnt = ccc.ccc2_rows_count(n_v, lo, hi)
    t = torch.full((cnt, 4), -7, dtype=torch.int32, device="cuda")
    c = torch.full((cnt, 4), -7.0, dtype=torch.float32, device="cuda")
    ccc.ccc2_tally_metric_rows(g, n_f, lo, hi, t, c, opts)
    torch.cuda.synchronize()
    p0 = oracle.pair_index(lo, lo + 1, n_v)
    assert_tally_equal(t.cpu().numpy(), et[p0:p0 + cnt], "fp4 rows")
    assert_ccc_close(c.cpu().numpy(), ec[p0:p0 + cnt], what="fp4 rows")
    # thresholded output: the hit set equals the oracle's above the threshold (pairs within
    # the tie band of the threshold may fall either way)
    thr = 0.155
    cap = 4096
    hits = torch.zeros(cap * 40, dtype=torch.uint8, device="cuda")
    n_hits = torch.zeros(1, dtype=torch.int64, device="cuda")
    ccc.ccc2_filter(g, n_f, thr, hits, cap, n_hits, opts)
    torch.cuda.synchronize()
    n = int(n_hits.item())
    rec = hits[:n * 40].cpu().numpy().view(np.int32).reshape(n, 10)
    got = {(int(r[0]), int(r[1])) for r in rec}
    mx = ec.max(axis=1)
    tie = np.abs(mx - thr) <= 1e-6 * thr
    keep = (mx > thr) & ~tie
    ii, jj = np.triu_indices(n_v, 1)
    want = set(zip(ii[keep].tolist(), jj[keep].tolist()))
    either = set(zip(ii[tie].tolist(), jj[tie].tolist()))
    assert want and want <= got <= want | either
    idx = oracle.pair_index(rec[:, 0].astype(np.int64), rec[:, 1].astype(np.int64), n_v)
    np.testing.assert_array_equal(rec[:, 2:6], et[idx])
    # phased output to pinned host memory
    wss = workspace(ccc.ccc2_stream_workspace_size(g, n_f, 4, opts0))
    optss = ccc.ccc_opts_default(workspace=wss, operand=E2M1)
    npairs = ccc.ccc2_count(n_v)
    ht = torch.empty((npairs, 4), dtype=torch.int32, pin_memory=True)
    hc = torch.empty((npairs, 4), dtype=torch.float32, pin_memory=True)
    ccc.ccc2_stream(g, n_f, 4, ht, hc, optss)
    torch.cuda.synchronize()
    assert_tally_equal(ht.numpy(), et, "fp4 stream")
    assert_ccc_close(hc.numpy(), ec, what="fp4 stream")


def test_fp4_where_not_built_is_refused():
    import torch

    import paper_1705_08213_gb300 as ccc
    geno = to_device(synth.panel_uniform(40, 100, seed=506))
    t = torch.empty((ccc.ccc2_count(40), 4), dtype=torch.int32, device="cuda")
    for tile in (1, 3):
        opts = ccc.ccc_opts_default(tile=tile, operand=E2M1)
        ws = workspace(ccc.ccc_workspace_size(geno, 100, opts, ccc.CCC_OP_2WAY))
        opts = ccc.ccc_opts_default(tile=tile, operand=E2M1, workspace=ws)
        with pytest.raises(ccc.CCCError) as e:
            ccc.ccc2_tally(geno, 100, t, opts)
        assert e.value.status == ccc.CCC_EUNSUPPORTED


# ---------------------------------------------------------------- 3-way (genotype classes)
#
# The sign-masked rows rho(x) s_j take the values 0, +-1, +-2 (e2m1 nibbles 0x0, 0x2, 0xA,
# 0x4, 0xC; a masked-out count is +-0), the compacted rows of the individuals with v_j missing
# 0, 1, 2; the wide class tiles are 128 SNPs i x 120 SNPs k here.


@pytest.mark.parametrize("n_f", [1, 255, 256, 257, 700])
@pytest.mark.parametrize("n_v", [3, 34, 130, 260])
def test_fp4_3way_edges_against_oracle(n_v, n_f):
    geno = synth.panel_uniform(n_v, n_f, seed=700 + n_v + n_f, p_missing=0.05, pad_seed=n_f + 3)
    t, c = run_3way(geno, n_f, 0, operand=E2M1)
    et, ec = oracle.ccc3_slabs(geno, n_f)
    assert_tally_equal(t, et, f"fp4 3-way tally n_v={n_v} n_f={n_f}")
    assert_ccc_close(c, ec, what=f"fp4 3-way ccc n_v={n_v} n_f={n_f}")


@pytest.mark.parametrize("norm", [0, 1])
def test_fp4_3way_equals_e4m3_bit_for_bit(norm):
    n_v, n_f = 300, 3000
    geno = synth.panel_hwe(n_v, n_f, seed=701, p_missing=0.02, pad_seed=13)
    t4, c4 = run_3way(geno, n_f, 0, norm=norm, operand=E2M1)
    t8, c8 = run_3way(geno, n_f, 0, norm=norm, operand=E4M3)
    np.testing.assert_array_equal(t4, t8)
    assert np.array_equal(c4.view(np.int32), c8.view(np.int32)), "CCC bits differ"
    # slab ranges, and the largest n_f of the wide tiles (D counts up to 4 n_f in 16 bits)
    for jb, je in ((0, 1), (117, 123), (150, 151), (240, 300)):
        t, c = run_3way(geno, n_f, 0, jb, je, norm=norm, operand=E2M1)
        et, ec = oracle.ccc3_slabs(geno, n_f, jb, je, norm=norm)
        assert_tally_equal(t, et, f"fp4 3-way slabs [{jb},{je})")
        assert_ccc_close(c, ec, what=f"fp4 3-way slabs [{jb},{je})")


def test_fp4_3way_missing_counts_and_the_width_limit():
    # SNPs with 0 .. 600 missing entries around the 256-individual compaction capacity,
    # and n_f = 16,383, the longest vectors of the wide tiles.
    n_f = 600
    counts = [0, 1, 127, 128, 255, 256, 257, 400, 600]
    g = synth.genotypes_uniform(8, 0, np.arange(3 * len(counts)), n_f, 0.0)
    rng = np.random.default_rng(14)
    for s_, m in enumerate(counts):
        g[3 * s_, rng.choice(n_f, size=m, replace=False)] = -1
    geno = synth.pack(synth.codes_from_genotypes(g), pad_seed=4)
    t, c = run_3way(geno, n_f, 0, operand=E2M1)
    et, ec = oracle.ccc3_slabs(geno, n_f)
    assert_tally_equal(t, et, "fp4 3-way missing counts")
    assert_ccc_close(c, ec, what="fp4 3-way missing counts")
    n_f = 16383
    geno = synth.pack(np.zeros((5, n_f), np.uint8))  # all (0,0): r^{000} = 8 n_f, D = 0
    t, _ = run_3way(geno, n_f, 0, operand=E2M1)
    assert np.all(t[:, 0] == 8 * n_f) and np.all(t[:, 1:] == 0)
    geno = synth.panel_hwe(40, n_f, seed=702, p_missing=0.02)
    t, c = run_3way(geno, n_f, 0, operand=E2M1)
    et, ec = oracle.ccc3_slabs(geno, n_f)
    assert_tally_equal(t, et, "fp4 3-way n_f = 16,383")
    assert_ccc_close(c, ec, what="fp4 3-way n_f = 16,383")


def test_fp4_3way_where_not_built_is_refused():
    import torch

    import paper_1705_08213_gb300 as ccc
    for n_f, tile in ((16384, 0), (300, 1), (300, 2)):
        geno = to_device(synth.panel_uniform(10, n_f, seed=703))
        nt = ccc.ccc3_count(10, 0, 10)
        t = torch.empty((nt, 8), dtype=torch.int32, device="cuda")
        opts = ccc.ccc_opts_default(tile=tile, operand=E2M1)
        ws = workspace(ccc.ccc_workspace_size(geno, n_f, opts, ccc.CCC_OP_3WAY))
        opts = ccc.ccc_opts_default(tile=tile, operand=E2M1, workspace=ws)
        with pytest.raises(ccc.CCCError) as e:
            ccc.ccc3_tally(geno, n_f, 0, 10, t, opts)
        assert e.value.status == ccc.CCC_EUNSUPPORTED
