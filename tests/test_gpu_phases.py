"""GPU 2-way phases: row-range calls and phased output to pinned host memory."""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_ccc_close, assert_tally_equal, run_2way, run_3way, to_device, workspace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


@pytest.mark.parametrize("path", [0, 1])
def test_row_ranges_equal_slices_of_the_full_result(path):
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 333, 700
    geno = synth.panel_hwe(n_v, n_f, seed=61, p_missing=0.02, pad_seed=1)
    full_t, full_c = run_2way(geno, n_f, path)
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(full_t, et, "full")
    g = to_device(geno)
    opts = ccc.ccc_opts_default(path=path)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(path=path, workspace=ws)
    for i0, i1 in ((0, 64), (64, 200), (3, 77), (200, 333), (332, 333), (0, 333), (150, 150)):
        cnt = ccc.ccc2_rows_count(n_v, i0, i1)
        t = torch.full((max(cnt, 1), 4), -7, dtype=torch.int32, device="cuda")
        c = torch.full((max(cnt, 1), 4), -7.0, dtype=torch.float32, device="cuda")
        ccc.ccc2_tally_metric_rows(g, n_f, i0, i1, t, c, opts)
        torch.cuda.synchronize()
        lo = ccc.ccc2_rows_count(n_v, 0, i0)
        np.testing.assert_array_equal(t[:cnt].cpu().numpy(), full_t[lo:lo + cnt])
        np.testing.assert_array_equal(c[:cnt].cpu().numpy(), full_c[lo:lo + cnt])
        if cnt == 0:
            assert int(t[0, 0]) == -7  # nothing written


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("n_phases", [2, 3, 7])
def test_stream_to_pinned_host(path, n_phases):
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 700, 1500
    geno = synth.panel_hwe(n_v, n_f, seed=62, p_missing=0.01)
    et, ec = oracle.ccc2_all(geno, n_f)
    g = to_device(geno)
    opts = ccc.ccc_opts_default(path=path)
    ws = workspace(ccc.ccc2_stream_workspace_size(g, n_f, n_phases, opts))
    opts = ccc.ccc_opts_default(path=path, workspace=ws)
    npairs = ccc.ccc2_count(n_v)
    ht = torch.full((npairs, 4), -7, dtype=torch.int32).pin_memory()
    hc = torch.full((npairs, 4), -7.0, dtype=torch.float32).pin_memory()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ccc.ccc2_stream(g, n_f, n_phases, ht, hc, opts, stream=s)
    s.synchronize()
    assert ccc.ccc_status(opts, stream=s) == ccc.CCC_OK
    assert_tally_equal(ht.numpy(), et, "streamed tallies")
    assert_ccc_close(hc.numpy(), ec, what="streamed CCC")
    ht2 = torch.zeros((npairs, 4), dtype=torch.int32).pin_memory()
    with torch.cuda.stream(s):
        ccc.ccc2_stream(g, n_f, n_phases, ht2, None, opts, stream=s)
    s.synchronize()
    assert_tally_equal(ht2.numpy(), et, "streamed tallies only")


@pytest.mark.parametrize("path", [(0, 0), (0, 1), (1, 0)])
@pytest.mark.parametrize("n_phases", [2, 5])
def test_stream3_to_pinned_host(path, n_phases):
    """ccc3_stream: all triples phase by phase into pinned host arrays equal the oracle
    (tensor cores by genotype classes and by masked operands, popcount)."""
    import torch

    import paper_1705_08213_gb300 as ccc
    path, tile = path
    n_v, n_f = 150, 700
    geno = synth.panel_hwe(n_v, n_f, seed=63, p_missing=0.02)
    et, ec = oracle.ccc3_slabs(geno, n_f)
    g = to_device(geno)
    opts = ccc.ccc_opts_default(path=path, tile=tile)
    ws = workspace(ccc.ccc3_stream_workspace_size(g, n_f, n_phases, opts))
    opts = ccc.ccc_opts_default(path=path, workspace=ws, tile=tile)
    nt = ccc.ccc3_count(n_v, 0, n_v)
    ht = torch.full((nt, 8), -7, dtype=torch.int32).pin_memory()
    hc = torch.full((nt, 8), -7.0, dtype=torch.float32).pin_memory()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ccc.ccc3_stream(g, n_f, n_phases, ht, hc, opts, stream=s)
    s.synchronize()
    assert ccc.ccc_status(opts, stream=s) == ccc.CCC_OK
    assert_tally_equal(ht.numpy(), et, "streamed 3-way tallies")
    assert_ccc_close(hc.numpy(), ec, what="streamed 3-way CCC")
    ht2 = torch.zeros((nt, 8), dtype=torch.int32).pin_memory()
    with torch.cuda.stream(s):
        ccc.ccc3_stream(g, n_f, n_phases, ht2, None, opts, stream=s)
    s.synchronize()
    assert_tally_equal(ht2.numpy(), et, "streamed 3-way tallies only")


@pytest.mark.parametrize("kind", [2, 3])
def test_field_slices_sum_to_the_full_tallies(kind):
    """The n_pf split on one device: tallies over slices of the individuals (views of the packed
    panel) sum to the full tallies; CCC values from the summed tallies and the whole panel's
    counts equal the fused call's bit for bit."""
    import torch

    import paper_1705_08213_gb300 as ccc
    from paper_1705_08213_gb300 import shard
    n_v, n_f = (700, 3000) if kind == 2 else (120, 1500)
    geno = synth.panel_hwe(n_v, n_f, seed=77, p_missing=0.02)
    g = to_device(geno)
    op = ccc.CCC_OP_2WAY if kind == 2 else ccc.CCC_OP_3WAY
    opts = ccc.ccc_opts_default()
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, op))
    opts = ccc.ccc_opts_default(workspace=ws)
    rows = ccc.ccc2_count(n_v) if kind == 2 else ccc.ccc3_count(n_v, 0, n_v)
    width = 4 if kind == 2 else 8
    total = torch.zeros((rows, width), dtype=torch.int32, device="cuda")
    part = torch.empty_like(total)
    for r in range(3):
        q0, q1 = shard.field_range(n_f, 3, r)
        if q0 == q1:
            continue
        if kind == 2:
            shard.field_tally2(g, n_f, q0, q1, part, opts)
        else:
            shard.field_tally3(g, n_f, q0, q1, 0, n_v, part, opts)
        total += part
    t_full, c_full = (run_2way(geno, n_f, 0) if kind == 2 else run_3way(geno, n_f, 0))
    np.testing.assert_array_equal(total.cpu().numpy(), t_full)
    counts = torch.zeros((n_v, 3), dtype=torch.int32, device="cuda")
    ccc.ccc_allele_counts(g, n_f, counts)
    wsm = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_METRIC))
    optm = ccc.ccc_opts_default(workspace=wsm)
    out = torch.empty((rows, width), dtype=torch.float32, device="cuda")
    if kind == 2:
        ccc.ccc2_metric(total, counts, n_v, optm, out)
    else:
        ccc.ccc3_metric(total, counts, n_v, 0, n_v, optm, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), c_full)
