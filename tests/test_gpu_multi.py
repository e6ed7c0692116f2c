"""GPU parity of the multi-allelic 2-way path (markers with s states) against the oracle.

Tallies must equal the oracle's exactly and CCC values agree within 1e-6
relative, for every state count 2..15, both normalisations, ragged sizes that
span several 256-row blocks and K stages, the degenerate cases, and sampled
rows of the full-size workload.  s = 2 must reproduce the biallelic kernel bit
for bit.  With s <= 8 the automatic operands are e2m1 (256 x 192 tiles of
8 PW x 6 PW markers, PW = floor(32 / s)); they must equal the e4m3 operands bit
for bit.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import (assert_ccc_close, assert_tally_equal, run_2way, run_multi,
                            to_device_bytes, workspace)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


# (s, n_v, n_f): n_v spans several 256-row blocks (8 floor(32/s) markers each) with a ragged
# last block; n_f is ragged against the 128-individual K stage.
SHAPES = [(2, 300, 1000), (3, 170, 777), (4, 100, 1000), (5, 70, 513), (6, 61, 300),
          (7, 40, 1201), (8, 70, 257), (9, 50, 129), (10, 30, 640), (11, 33, 333),
          (13, 20, 100), (15, 37, 1025)]


@pytest.mark.parametrize("s,n_v,n_f", SHAPES, ids=[f"s{s}-{v}x{f}" for s, v, f in SHAPES])
@pytest.mark.parametrize("norm", [0, 1])
def test_against_oracle(s, n_v, n_f, norm):
    g = synth.panel_multi(n_v, n_f, s, seed=40 + s, p_missing=0.03, pad_seed=7)
    t, c = run_multi(g, n_f, s, norm=norm)
    et, ec = oracle.ccc2_multi_all(g, n_f, s, norm=norm)
    assert_tally_equal(t, et, f"s={s}")
    assert_ccc_close(c, ec, what=f"s={s}")


@pytest.mark.parametrize("s", [3, 4, 8, 15])
def test_metric_from_tallies_equals_fused(s):
    n_v, n_f = 90, 700
    g = synth.panel_multi(n_v, n_f, s, seed=60 + s, p_missing=0.05)
    for norm in (0, 1):
        t1, c1 = run_multi(g, n_f, s, norm=norm, fused=True)
        t2, c2 = run_multi(g, n_f, s, norm=norm, fused=False)
        np.testing.assert_array_equal(t1, t2)
        np.testing.assert_array_equal(c1, c2)


@pytest.mark.parametrize("s", [2, 5, 15])
def test_counts_against_oracle(s):
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 77, 1111
    g = synth.panel_multi(n_v, n_f, s, seed=70 + s, p_missing=0.1, pad_seed=9)
    counts = torch.full((n_v, s + 1), -1, dtype=torch.int32, device="cuda")
    ccc.ccc_multi_counts(to_device_bytes(g), n_f, s, counts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(counts.cpu().numpy(), oracle.multi_counts(g, n_f, s))


@pytest.mark.parametrize("norm", [0, 1])
def test_two_states_equal_biallelic_kernel(norm):
    n_v, n_f = 530, 2000
    words = synth.panel_hwe(n_v, n_f, seed=21, p_missing=0.02)
    g = synth.multi_from_biallelic(words, n_f)
    tm, cm = run_multi(g, n_f, 2, norm=norm)
    t2, c2 = run_2way(words, n_f, 0, norm=norm)
    np.testing.assert_array_equal(tm, t2)
    np.testing.assert_array_equal(cm, c2)


def test_degenerate_cases():
    s = 4
    # one marker: no pairs, nothing written, status OK
    g1 = synth.panel_multi(1, 50, s, seed=1)
    t, c = run_multi(g1, 50, s)
    assert t.shape == (0, 16)
    # two markers, one individual
    g2 = synth.panel_multi(2, 1, s, seed=2, p_missing=0.0)
    t, c = run_multi(g2, 1, s)
    et, ec = oracle.ccc2_multi_all(g2, 1, s)
    assert_tally_equal(t, et, "n_f=1")
    assert_ccc_close(c, ec, what="n_f=1")
    # a marker with every entry missing, and one with every entry missing but the padding
    g3 = synth.panel_multi(40, 300, s, seed=3, p_missing=0.02, pad_seed=5)
    g3[7, :300] = 0xFF
    g3[8, :300] = 0x4F  # low nibble 15 >= s: missing
    t, c = run_multi(g3, 300, s)
    et, ec = oracle.ccc2_multi_all(g3, 300, s)
    assert_tally_equal(t, et, "all missing")
    assert_ccc_close(c, ec, what="all missing")
    idx = oracle.pair_index(np.array([0, 7, 7, 8]), np.array([7, 8, 39, 20]), 40)
    assert np.all(t[idx] == 0) and np.all(c[idx] == 0)


def test_long_vectors_exact():
    """Tallies up to 4 n_f: identical homozygous markers over 300,000 individuals."""
    s, n_v, n_f = 3, 20, 300000
    g = np.zeros((n_v, synth.multi_default_ld(n_f)), np.uint8)
    g[:, :n_f] = 0x22  # state (2, 2) everywhere
    g[5, :n_f:2] = 0x10  # every other entry (0, 1)
    t, c = run_multi(g, n_f, s)
    et, ec = oracle.ccc2_multi_all(g, n_f, s)
    assert_tally_equal(t, et, "long")
    assert_ccc_close(c, ec, what="long")
    assert t.max() == 4 * n_f


def test_full_size_workload_sampled_rows():
    """The multi-allelic bench workload: 10,000 markers x 16,384 individuals, s = 4, 1% missing;
    three full rows of the triangle against the oracle, with the launch bench.py times."""
    import torch

    import paper_1705_08213_gb300 as ccc
    s, n_v, n_f = 4, 10000, 16384
    g = synth.panel_multi(n_v, n_f, s, seed=6, p_missing=0.01)
    dg = to_device_bytes(g)
    npairs = ccc.ccc2_count(n_v)
    opts = ccc.ccc_opts_default()
    ws = workspace(ccc.ccc_multi_workspace_size(dg, n_f, s, opts))
    opts = ccc.ccc_opts_default(workspace=ws)
    tally = torch.empty((npairs, s * s), dtype=torch.int32, device="cuda")
    out = torch.empty((npairs, s * s), dtype=torch.float32, device="cuda")
    ccc.ccc2_multi_tally_metric(dg, n_f, s, tally, out, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    rows = np.array([0, 4321, n_v - 2])
    et, ec = oracle.ccc2_multi_rows(g, n_f, s, rows)
    idx = np.concatenate([oracle.pair_index(i, np.arange(i + 1, n_v), n_v) for i in rows])
    it = torch.from_numpy(idx).cuda()
    assert_tally_equal(tally[it].cpu().numpy(), et, "full-size rows")
    assert_ccc_close(out[it].cpu().numpy(), ec, what="full-size rows")


def test_tile_order_groups_agree():
    s, n_v, n_f = 5, 400, 600
    g = synth.panel_multi(n_v, n_f, s, seed=80, p_missing=0.02)
    t0, c0 = run_multi(g, n_f, s)
    for group in (1, 3, 16):
        t1, c1 = run_multi(g, n_f, s, group=group)
        np.testing.assert_array_equal(t1, t0)
        np.testing.assert_array_equal(c1, c0)


def test_workspace_too_small_is_refused():
    import torch

    import paper_1705_08213_gb300 as ccc
    s, n_v, n_f = 4, 50, 200
    g = to_device_bytes(synth.panel_multi(n_v, n_f, s, seed=81))
    opts = ccc.ccc_opts_default()
    need = ccc.ccc_multi_workspace_size(g, n_f, s, opts)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    opts = ccc.ccc_opts_default(workspace=ws)
    opts.workspace_bytes = need - 1
    tally = torch.full((ccc.ccc2_count(n_v), s * s), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc2_multi_tally(g, n_f, s, tally, opts)
    assert e.value.status == ccc.CCC_ENOSPACE
    torch.cuda.synchronize()
    assert bool((tally == -7).all())  # nothing was written


def test_cuda_graph_capture_and_replay():
    import torch

    import paper_1705_08213_gb300 as ccc
    s, n_v, n_f = 3, 300, 500
    gm = synth.panel_multi(n_v, n_f, s, seed=82, p_missing=0.03)
    g = to_device_bytes(gm)
    opts = ccc.ccc_opts_default()
    ws = torch.empty(ccc.ccc_multi_workspace_size(g, n_f, s, opts), dtype=torch.uint8, device="cuda")
    opts = ccc.ccc_opts_default(workspace=ws)
    npairs = ccc.ccc2_count(n_v)
    tally = torch.zeros((npairs, s * s), dtype=torch.int32, device="cuda")
    out = torch.zeros((npairs, s * s), dtype=torch.float32, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ccc.ccc2_multi_tally_metric(g, n_f, s, tally, out, opts, stream=st)  # first call outside
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        ccc.ccc2_multi_tally_metric(g, n_f, s, tally, out, opts, stream=st)
    tally.zero_()
    out.zero_()
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    et, ec = oracle.ccc2_multi_all(gm, n_f, s)
    assert_tally_equal(tally.cpu().numpy(), et, "graph replay")
    assert_ccc_close(out.cpu().numpy(), ec, what="graph replay")


@pytest.mark.parametrize("s", [3, 4, 11])
def test_row_ranges_equal_slices_of_the_full_call(s):
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 260, 700
    gm = synth.panel_multi(n_v, n_f, s, seed=90 + s, p_missing=0.03)
    t_full, c_full = run_multi(gm, n_f, s)
    g = to_device_bytes(gm)
    opts = ccc.ccc_opts_default()
    ws = torch.empty(ccc.ccc_multi_workspace_size(g, n_f, s, opts), dtype=torch.uint8, device="cuda")
    opts = ccc.ccc_opts_default(workspace=ws)
    step = 8 * (32 // s)
    for i0, i1 in ((0, step), (step, 3 * step), (5, 77), (n_v - 3, n_v), (100, 100)):
        i1 = min(i1, n_v)
        cnt = ccc.ccc2_rows_count(n_v, i0, i1)
        t = torch.full((max(cnt, 1), s * s), -7, dtype=torch.int32, device="cuda")
        c = torch.full((max(cnt, 1), s * s), -7.0, dtype=torch.float32, device="cuda")
        ccc.ccc2_multi_tally_metric_rows(g, n_f, s, i0, i1, t, c, opts)
        torch.cuda.synchronize()
        assert ccc.ccc_status(opts) == ccc.CCC_OK
        p0 = ccc.ccc2_index(i0, i0 + 1, n_v) if cnt else 0
        np.testing.assert_array_equal(t[:cnt].cpu().numpy(), t_full[p0:p0 + cnt])
        np.testing.assert_array_equal(c[:cnt].cpu().numpy(), c_full[p0:p0 + cnt])


@pytest.mark.parametrize("n_phases", [2, 5])
def test_stream_to_pinned_host(n_phases):
    import torch

    import paper_1705_08213_gb300 as ccc
    s, n_v, n_f = 4, 700, 900
    gm = synth.panel_multi(n_v, n_f, s, seed=95, p_missing=0.02)
    t_full, c_full = run_multi(gm, n_f, s)
    g = to_device_bytes(gm)
    opts = ccc.ccc_opts_default()
    ws = torch.empty(ccc.ccc2_multi_stream_workspace_size(g, n_f, s, n_phases, opts),
                     dtype=torch.uint8, device="cuda")
    opts = ccc.ccc_opts_default(workspace=ws)
    npairs = ccc.ccc2_count(n_v)
    ht = torch.full((npairs, s * s), -7, dtype=torch.int32, pin_memory=True)
    hc = torch.full((npairs, s * s), -7.0, dtype=torch.float32, pin_memory=True)
    ccc.ccc2_multi_stream(g, n_f, s, n_phases, ht, hc, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    np.testing.assert_array_equal(ht.numpy(), t_full)
    np.testing.assert_array_equal(hc.numpy(), c_full)
    # tallies only
    ht2 = torch.full((npairs, s * s), -7, dtype=torch.int32, pin_memory=True)
    ccc.ccc2_multi_stream(g, n_f, s, n_phases, ht2, None, opts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ht2.numpy(), t_full)


E4M3, E2M1 = 1, 2


@pytest.mark.parametrize("s", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("norm", [0, 1])
def test_fp4_equals_e4m3_bit_for_bit(s, norm):
    pw = 32 // s
    n_v, n_f = 6 * pw * 3 + 8 * pw + 5, 700
    g = synth.panel_multi(n_v, n_f, s, seed=140 + s, p_missing=0.04, pad_seed=9)
    t4, c4 = run_multi(g, n_f, s, norm=norm, operand=E2M1, split=1)
    t8, c8 = run_multi(g, n_f, s, norm=norm, operand=E4M3, split=1)
    np.testing.assert_array_equal(t4, t8)
    assert np.array_equal(c4.view(np.int32), c8.view(np.int32)), "CCC bits differ"


# e2m1 tiles: marker counts around multiples of the 6 PW column block and the 8 PW row block,
# individual counts around the 256-entry K stage
FP4_EDGES = [(4, 47, 255), (4, 48, 256), (4, 49, 257), (4, 64, 513), (4, 97, 300),
             (3, 59, 256), (3, 60, 511), (3, 81, 700), (7, 23, 129), (7, 25, 1000),
             (8, 24, 257), (2, 95, 600), (2, 130, 1)]


@pytest.mark.parametrize("s,n_v,n_f", FP4_EDGES, ids=[f"s{s}-{v}x{f}" for s, v, f in FP4_EDGES])
def test_fp4_tile_edges_against_oracle(s, n_v, n_f):
    g = synth.panel_multi(n_v, n_f, s, seed=160 + n_v, p_missing=0.05, pad_seed=n_f)
    t, c = run_multi(g, n_f, s, operand=E2M1)
    et, ec = oracle.ccc2_multi_all(g, n_f, s)
    assert_tally_equal(t, et, f"fp4 s={s} {n_v}x{n_f}")
    assert_ccc_close(c, ec, what=f"fp4 s={s} {n_v}x{n_f}")


def test_fp4_long_vectors_unsplit():
    """One e2m1 accumulator per entry summing all n_f: tallies up to 4 n_f."""
    s, n_v, n_f = 3, 20, 300000
    g = np.zeros((n_v, synth.multi_default_ld(n_f)), np.uint8)
    g[:, :n_f] = 0x22
    g[5, :n_f:2] = 0x10
    t, c = run_multi(g, n_f, s, operand=E2M1, split=1)
    et, ec = oracle.ccc2_multi_all(g, n_f, s)
    assert_tally_equal(t, et, "fp4 long")
    assert_ccc_close(c, ec, what="fp4 long")
    assert t.max() == 4 * n_f


def test_fp4_refused_where_not_built():
    import torch

    import paper_1705_08213_gb300 as ccc
    s, n_v, n_f = 9, 20, 300
    g = synth.panel_multi(n_v, n_f, s, seed=170)
    dg = to_device_bytes(g)
    opts = ccc.ccc_opts_default()
    ws = workspace(ccc.ccc_multi_workspace_size(dg, n_f, s, opts))
    npairs = ccc.ccc2_count(n_v)
    tally = torch.zeros((npairs, s * s), dtype=torch.int32, device="cuda")
    out = torch.zeros((npairs, s * s), dtype=torch.float32, device="cuda")
    for kw in (dict(operand=E2M1), dict(operand=E2M1, split=4)):
        opts = ccc.ccc_opts_default(workspace=ws)
        opts.operand = kw["operand"]
        opts.split = kw.get("split", 0)
        with pytest.raises(ccc.CCCError) as e:
            ccc.ccc2_multi_tally_metric(dg, n_f, s, tally, out, opts)
        assert e.value.status == ccc.CCC_EUNSUPPORTED
    # s <= 8 with an explicit K split: e2m1 is not built there either
    g4 = synth.panel_multi(n_v, n_f, 4, seed=171)
    dg4 = to_device_bytes(g4)
    ws4 = workspace(ccc.ccc_multi_workspace_size(dg4, n_f, 4, ccc.ccc_opts_default()))
    opts = ccc.ccc_opts_default(workspace=ws4)
    opts.operand = E2M1
    opts.split = 2
    t4 = torch.zeros((npairs, 16), dtype=torch.int32, device="cuda")
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc2_multi_tally(dg4, n_f, 4, t4, opts)
    assert e.value.status == ccc.CCC_EUNSUPPORTED
