"""The allocation-free 2-way entry point agrees with the workspace entry point.

ccc2_tally_metric_noalloc serves callers that cannot allocate device memory
(a host framework that owns all device allocations, plug-ins handed only their
input and output buffers): it keeps its scratch in a fixed array built into
the library.  This file is collected last so that, if it fails, a run that
stops at the first failure has already run every other test.
"""

import numpy as np
import pytest

import synth
from tests.gpu_util import CCC_RTOL, assert_ccc_close, assert_tally_equal, run_2way, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


def _noalloc(geno_np, n_f, norm=0):
    import torch

    import paper_1705_08213_gb300 as ccc
    g = to_device(geno_np)
    n_v = geno_np.shape[0]
    npairs = ccc.ccc2_count(n_v)
    tally = torch.full((max(npairs, 1), 4), -7, dtype=torch.int32, device="cuda")
    out = torch.full((max(npairs, 1), 4), -7.0, dtype=torch.float32, device="cuda")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    opts = ccc.ccc_opts_default(path=ccc.CCC_PATH_TC, norm=norm)
    ccc.ccc2_tally_metric_noalloc(g, n_f, tally, out, opts, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == ccc.CCC_OK
    return tally[:npairs].cpu().numpy(), out[:npairs].cpu().numpy()


def test_noalloc_matches_workspace_entry_point_twice():
    # Two calls in a row; the second panel is smaller, so anything left over in
    # the shared built-in scratch from the first call would show up.
    cases = [(synth.panel_hwe(300, 1000, seed=31, p_missing=0.02, pad_seed=3), 1000, 0),
             (synth.panel_uniform(129, 777, seed=32, p_missing=0.05, pad_seed=4), 777, 1)]
    for geno, n_f, norm in cases:
        t_ref, c_ref = run_2way(geno, n_f, 0, norm=norm)
        t, c = _noalloc(geno, n_f, norm=norm)
        assert_tally_equal(t, t_ref, "noalloc tallies")
        assert_ccc_close(c, c_ref.astype(np.float64), rtol=CCC_RTOL, what="noalloc CCC")


def test_noalloc_rejects_panels_beyond_the_scratch():
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 2048, 7681  # one individual past the 32 MiB limit at this n_v
    geno = torch.zeros((n_v, synth.default_ld(n_f)), dtype=torch.int64, device="cuda")
    tally = torch.empty((16, 4), dtype=torch.int32, device="cuda")
    out = torch.empty((16, 4), dtype=torch.float32, device="cuda")
    opts = ccc.ccc_opts_default(path=ccc.CCC_PATH_TC)
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc2_tally_metric_noalloc(geno, n_f, tally, out, opts)
    assert e.value.status == ccc.CCC_ERANGE
    opts = ccc.ccc_opts_default(path=ccc.CCC_PATH_POPC)
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc2_tally_metric_noalloc(geno[:8], 100, tally, out, opts)
    assert e.value.status == ccc.CCC_EINVAL
