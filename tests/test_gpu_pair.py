"""GPU parity of the 2-way tensor-core kernel on SM pairs (256 x 256 tiles, cta_group::2)."""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_ccc_close, assert_tally_equal, run_2way

pytestmark = pytest.mark.gpu

PAIR = 2


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


@pytest.mark.parametrize("n_v,n_f", [(2, 1), (3, 33), (64, 129), (127, 1000), (128, 128),
                                     (129, 257), (255, 64), (256, 1024), (300, 777), (600, 300)])
def test_pair_tiles_against_oracle(n_v, n_f):
    geno = synth.panel_uniform(n_v, n_f, seed=700 + n_v, p_missing=0.03, pad_seed=n_v)
    t, c = run_2way(geno, n_f, 0, tile=PAIR)
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t, et, f"pair n_v={n_v} n_f={n_f}")
    assert_ccc_close(c, ec, what=f"pair n_v={n_v} n_f={n_f}")


def test_pair_equals_single_sm_tiles_with_long_k():
    geno = synth.panel_hwe(1000, 20000, seed=71, p_missing=0.01)
    t1, c1 = run_2way(geno, 20000, 0, tile=1)
    t2, c2 = run_2way(geno, 20000, 0, tile=PAIR)
    np.testing.assert_array_equal(t1, t2)
    np.testing.assert_array_equal(c1, c2)
    et, ec = oracle.ccc2_rows(geno, 20000, np.array([0, 511, 998]))
    idx = np.concatenate([oracle.pair_index(i, np.arange(i + 1, 1000), 1000) for i in (0, 511, 998)])
    assert_tally_equal(t2[idx], et, "pair rows")


def test_pair_row_ranges_and_stream():
    import torch

    import paper_1705_08213_gb300 as ccc
    from tests.gpu_util import to_device, workspace
    n_v, n_f = 700, 2000
    geno = synth.panel_hwe(n_v, n_f, seed=72, p_missing=0.01)
    full_t, full_c = run_2way(geno, n_f, 0, tile=1)
    g = to_device(geno)
    opts = ccc.ccc_opts_default(tile=PAIR)
    ws = workspace(ccc.ccc2_stream_workspace_size(g, n_f, 5, opts))
    opts = ccc.ccc_opts_default(workspace=ws, tile=PAIR)
    for i0, i1 in ((0, 128), (100, 400), (640, 700)):
        cnt = ccc.ccc2_rows_count(n_v, i0, i1)
        t = torch.empty((cnt, 4), dtype=torch.int32, device="cuda")
        c = torch.empty((cnt, 4), dtype=torch.float32, device="cuda")
        ccc.ccc2_tally_metric_rows(g, n_f, i0, i1, t, c, opts)
        torch.cuda.synchronize()
        lo = ccc.ccc2_rows_count(n_v, 0, i0)
        np.testing.assert_array_equal(t.cpu().numpy(), full_t[lo:lo + cnt])
    npairs = ccc.ccc2_count(n_v)
    ht = torch.empty((npairs, 4), dtype=torch.int32).pin_memory()
    hc = torch.empty((npairs, 4), dtype=torch.float32).pin_memory()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ccc.ccc2_stream(g, n_f, 5, ht, hc, opts, stream=s)
    s.synchronize()
    np.testing.assert_array_equal(ht.numpy(), full_t)
    np.testing.assert_array_equal(hc.numpy(), full_c)
