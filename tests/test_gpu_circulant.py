"""The block-circulant 2-way decomposition (Sec. 4, n_pv axis) through the C ABI.

Every rank's block row is computed on this one GPU in turn, each from a local
panel that holds only that rank's vector blocks (ccc2_tally_metric_rows over
its own block's rows); scattered to the global pair order, the union equals
the whole-panel call: tallies bit for bit, CCC values within 1e-6 of the
oracle (a transposed pair's values are the same products in another order).
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_ccc_close, assert_tally_equal, run_2way, to_device, workspace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_circulant_block_rows_reassemble_the_triangle(world):
    import torch

    import paper_1705_08213_gb300 as ccc
    from paper_1705_08213_gb300 import shard
    n_v, n_f = 700, 3000
    geno = synth.panel_hwe(n_v, n_f, seed=600 + world, p_missing=0.02)
    t_full, c_full = run_2way(geno, n_f, 0)
    g = to_device(geno)
    npairs = ccc.ccc2_count(n_v)
    t = np.full((npairs, 4), -7, np.int64)
    c = np.full((npairs, 4), np.nan, np.float64)
    for rank in range(world):
        plan = shard.circulant_plan(n_v, world, rank)
        local = shard.circulant_local_panel(g, plan).contiguous()
        lo, hi = plan["rows"]
        cnt = ccc.ccc2_rows_count(local.shape[0], lo, hi)
        if cnt == 0:
            continue
        opts = ccc.ccc_opts_default()
        ws = workspace(ccc.ccc_workspace_size(local, n_f, opts, ccc.CCC_OP_2WAY))
        opts = ccc.ccc_opts_default(workspace=ws)
        tl = torch.full((cnt, 4), -7, dtype=torch.int32, device="cuda")
        cl = torch.full((cnt, 4), -7.0, dtype=torch.float32, device="cuda")
        shard.circulant_block_row(local, n_f, plan, tl, cl, opts)
        torch.cuda.synchronize()
        assert ccc.ccc_status(opts) == ccc.CCC_OK
        idx, ts, cs = shard.circulant_scatter(plan, tl.cpu().numpy(), cl.cpu().numpy())
        assert np.all(t[idx, 0] == -7), "a pair computed twice"
        t[idx] = ts
        c[idx] = cs
    assert_tally_equal(t, t_full, f"block-circulant tallies, {world} ranks")
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t, et, "block-circulant tallies vs oracle")
    assert_ccc_close(c, ec, what=f"block-circulant CCC, {world} ranks")
