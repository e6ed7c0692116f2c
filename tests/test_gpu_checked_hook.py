"""The index checks of the bounds-checking build catch what they must.

tests/test_gpu_checked.py runs this file in a child process whose CCC_LIBRARY is the
library built with -DCCC_BOUNDS_CHECK; under the normal build it is skipped.

ccc_checked_shrink_outputs(n) (include/ccc_checked.h) makes later calls tell their kernels
that the output arrays hold n fewer entries than they do.  The stores of the last n
entries must then be caught by the kernels' index checks: the call's status is
CCC_EBOUNDS, those entries keep the values they had, and every other entry equals the
oracle's.  Every real access stays inside the arrays.  Covered: the 2-way tensor-core
kernels (one SM, SM pairs, codes expanded in shared memory, K split), the 2-way popcount
kernel, the 3-way genotype-class, masked-operand and popcount kernels, and the s-state
kernel.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_ccc_close, assert_tally_equal, to_device, to_device_bytes, workspace

pytestmark = pytest.mark.gpu

SHRINK = 5


@pytest.fixture(scope="module", autouse=True)
def _checked_build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1705_08213_gb300 as ccc
    if not ccc.lib_path.endswith("libccc_checked.so"):
        pytest.skip("needs the bounds-checking build (CCC_LIBRARY)")
    yield
    ccc.ccc_checked_shrink_outputs(0)


def _shrunk(call, opts):
    import torch

    import paper_1705_08213_gb300 as ccc
    ccc.ccc_checked_shrink_outputs(SHRINK)
    try:
        call()
        torch.cuda.synchronize()
    finally:
        ccc.ccc_checked_shrink_outputs(0)
    return ccc.ccc_status(opts)


@pytest.mark.parametrize("path,tile,split", [(0, 1, 1), (0, 2, 1), (0, 3, 1), (0, 2, 4), (0, 3, 4),
                                             (1, 0, 1)])
def test_2way_last_pairs_are_caught(path, tile, split):
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 300, 1000
    geno = synth.panel_hwe(n_v, n_f, seed=120 + tile, p_missing=0.02)
    g = to_device(geno)
    opts = ccc.ccc_opts_default(path=path, tile=tile)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(path=path, tile=tile, workspace=ws)
    opts.split = split
    npairs = ccc.ccc2_count(n_v)
    t = torch.full((npairs, 4), -7, dtype=torch.int32, device="cuda")
    c = torch.full((npairs, 4), -7.0, dtype=torch.float32, device="cuda")
    st = _shrunk(lambda: ccc.ccc2_tally_metric(g, n_f, t, c, opts), opts)
    assert st == ccc.CCC_EBOUNDS
    t, c = t.cpu().numpy(), c.cpu().numpy()
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t[:-SHRINK], et[:-SHRINK], "pairs before the hidden ones")
    assert_ccc_close(c[:-SHRINK], ec[:-SHRINK], what="pairs before the hidden ones")
    # K split: the output is zeroed first and the skipped partial sums leave zeros; the
    # CCC pass then runs over all pairs.  Otherwise both arrays keep the sentinel.
    assert np.all(t[-SHRINK:] == (0 if split > 1 else -7))
    if split == 1:
        assert np.all(c[-SHRINK:] == -7.0)
    # with the true lengths back, the next call clears the status and writes every pair
    t2 = torch.full((npairs, 4), -7, dtype=torch.int32, device="cuda")
    c2 = torch.full((npairs, 4), -7.0, dtype=torch.float32, device="cuda")
    ccc.ccc2_tally_metric(g, n_f, t2, c2, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    assert_tally_equal(t2.cpu().numpy(), et, "after the reset")


@pytest.mark.parametrize("path,tile", [(0, 0), (0, 1), (1, 0)])
def test_3way_last_triples_are_caught(path, tile):
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 40, 700
    geno = synth.panel_hwe(n_v, n_f, seed=130 + tile, p_missing=0.02)
    g = to_device(geno)
    opts = ccc.ccc_opts_default(path=path, tile=tile)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_3WAY))
    opts = ccc.ccc_opts_default(path=path, tile=tile, workspace=ws)
    nt = ccc.ccc3_count(n_v, 0, n_v)
    t = torch.full((nt, 8), -7, dtype=torch.int32, device="cuda")
    c = torch.full((nt, 8), -7.0, dtype=torch.float32, device="cuda")
    st = _shrunk(lambda: ccc.ccc3_tally_metric(g, n_f, 0, n_v, t, c, opts), opts)
    assert st == ccc.CCC_EBOUNDS
    t, c = t.cpu().numpy(), c.cpu().numpy()
    et, ec = oracle.ccc3_slabs(geno, n_f)
    assert_tally_equal(t[:-SHRINK], et[:-SHRINK], "triples before the hidden ones")
    assert_ccc_close(c[:-SHRINK], ec[:-SHRINK], what="triples before the hidden ones")
    assert np.all(t[-SHRINK:] == -7) and np.all(c[-SHRINK:] == -7.0)


def test_multi_last_pairs_are_caught():
    import torch

    import paper_1705_08213_gb300 as ccc
    s, n_v, n_f = 4, 150, 900
    gm = synth.panel_multi(n_v, n_f, s, seed=140, p_missing=0.02)
    g = to_device_bytes(gm)
    opts = ccc.ccc_opts_default()
    ws = workspace(ccc.ccc_multi_workspace_size(g, n_f, s, opts))
    opts = ccc.ccc_opts_default(workspace=ws)
    npairs = ccc.ccc2_count(n_v)
    t = torch.full((npairs, s * s), -7, dtype=torch.int32, device="cuda")
    c = torch.full((npairs, s * s), -7.0, dtype=torch.float32, device="cuda")
    st = _shrunk(lambda: ccc.ccc2_multi_tally_metric(g, n_f, s, t, c, opts), opts)
    assert st == ccc.CCC_EBOUNDS
    t, c = t.cpu().numpy(), c.cpu().numpy()
    et, ec = oracle.ccc2_multi_all(gm, n_f, s)
    assert_tally_equal(t[:-SHRINK], et[:-SHRINK], "pairs before the hidden ones")
    assert_ccc_close(c[:-SHRINK], ec[:-SHRINK], what="pairs before the hidden ones")
    assert np.all(t[-SHRINK:] == -7) and np.all(c[-SHRINK:] == -7.0)
